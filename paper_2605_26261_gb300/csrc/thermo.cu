// FTLM thermodynamic sums (step a6, Eq. 6-9), FP64 on the device.
//
// Every (sector image, chain, Ritz pair) contributes weight (D/R) w_k at energy
// E = theta_k - h S^z (Zeeman term -h S^z) and magnetization S^z; sectors with
// S^z > 0 also stand for -S^z when mirroring is on (identical spectra, Sec. 2).
// With E0 the lowest energy, one block per temperature forms
//   Z = sum b,  b = (D/R) w e^{-beta (E - E0)}       (Eq. 7, shifted by E0)
//   <E - E0> = sum b (E - E0) / Z,  Var(H) = sum b (E - E0 - <E - E0>)^2 / Z
//   <S^z> = sum b S^z / Z,  <(S^z)^2> = sum b (S^z)^2 / Z,
//   Var(S^z) = sum b (S^z - <S^z>)^2 / Z
// and C = beta^2 Var(H) (Eq. 8 moments, central form), chi = g^2 beta <(S^z)^2>
// at h = 0 (Eq. 9) and g^2 beta Var(S^z) otherwise.  The shift keeps e^{-beta E}
// finite at T = 0.01 and cancels in every ratio; the central second moment avoids
// the cancellation of <H^2> - <H>^2 at high T.  Sums use fixed-order block
// reductions, so results are reproducible.
#include <cmath>

#include "ftlm_internal.cuh"
#include "reduce.cuh"

namespace ftlm {

namespace {

constexpr int kThermoThreads = 256;

struct ThermoArgs {
    int ns, R, M, mirror;
    double g, h;
    const double *theta[FTLM_MAX_SECTORS];
    const double *weight[FTLM_MAX_SECTORS];
    const int *meff[FTLM_MAX_SECTORS];
    double wscale[FTLM_MAX_SECTORS];  // D / R
    double sz[FTLM_MAX_SECTORS];      // S^z
};

__device__ __forceinline__ double block_min(double v)
{
    __shared__ double sh[kThermoThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = sh[0];
    for (int i = 1; i < kThermoThreads / 32; ++i) r = fmin(r, sh[i]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ double bcast(double v)
{
    __shared__ double sh;
    if (threadIdx.x == 0) sh = v;
    __syncthreads();
    const double r = sh;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThermoThreads)
thermo_kernel(const ThermoArgs a, const double *__restrict__ T, double *E, double *C, double *chi,
              double *mag, double *Zs, double *E0s)
{
    const int per_sector = a.R * a.M;
    const int n = a.ns * per_sector;
    double emin = INFINITY;
    for (int i = threadIdx.x; i < n; i += kThermoThreads) {
        const int s = i / per_sector, rem = i - s * per_sector, r = rem / a.M, k = rem - r * a.M;
        if (k >= __ldg(a.meff[s] + r)) continue;
        const double th = __ldg(a.theta[s] + rem);
        emin = fmin(emin, th - a.h * a.sz[s]);
        if (a.mirror && a.sz[s] > 0.0) emin = fmin(emin, th + a.h * a.sz[s]);
    }
    const double E0 = block_min(emin);
    const double beta = 1.0 / T[blockIdx.x];

    double z = 0.0, s1 = 0.0, m1 = 0.0, m2 = 0.0;
    for (int i = threadIdx.x; i < n; i += kThermoThreads) {
        const int s = i / per_sector, rem = i - s * per_sector, r = rem / a.M, k = rem - r * a.M;
        if (k >= __ldg(a.meff[s] + r)) continue;
        const double th = __ldg(a.theta[s] + rem), w = __ldg(a.weight[s] + rem) * a.wscale[s];
        const int images = (a.mirror && a.sz[s] > 0.0) ? 2 : 1;
        for (int im = 0; im < images; ++im) {
            const double mz = im ? -a.sz[s] : a.sz[s];
            const double de = th - a.h * mz - E0;
            const double b = w * exp(-beta * de);
            z += b;
            s1 += b * de;
            m1 += b * mz;
            m2 += b * mz * mz;
        }
    }
    const double Z = bcast(block_sum<kThermoThreads>(z));
    const double e1 = bcast(block_sum<kThermoThreads>(s1)) / Z;
    const double M1 = bcast(block_sum<kThermoThreads>(m1)) / Z;
    const double M2 = bcast(block_sum<kThermoThreads>(m2)) / Z;

    double s2 = 0.0, v2 = 0.0;
    for (int i = threadIdx.x; i < n; i += kThermoThreads) {
        const int s = i / per_sector, rem = i - s * per_sector, r = rem / a.M, k = rem - r * a.M;
        if (k >= __ldg(a.meff[s] + r)) continue;
        const double th = __ldg(a.theta[s] + rem), w = __ldg(a.weight[s] + rem) * a.wscale[s];
        const int images = (a.mirror && a.sz[s] > 0.0) ? 2 : 1;
        for (int im = 0; im < images; ++im) {
            const double mz = im ? -a.sz[s] : a.sz[s];
            const double de = th - a.h * mz - E0;
            const double b = w * exp(-beta * de);
            const double dc = de - e1, dm = mz - M1;
            s2 += b * dc * dc;
            v2 += b * dm * dm;
        }
    }
    const double S2 = bcast(block_sum<kThermoThreads>(s2));
    const double V2 = block_sum<kThermoThreads>(v2);
    if (threadIdx.x == 0) {
        const int t = blockIdx.x;
        if (E) E[t] = E0 + e1;
        if (C) C[t] = beta * beta * (S2 / Z);
        if (chi) chi[t] = a.g * a.g * beta * (a.h == 0.0 ? M2 : V2 / Z);
        if (mag) mag[t] = M1;
        if (Zs) Zs[t] = Z;
        if (E0s) E0s[t] = E0;
    }
}

}  // namespace

}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_thermo(int n_sectors, const int *two_sz, const uint64_t *dims, int R, int M,
                                   const double *const *theta, const double *const *weight,
                                   const int *const *m_eff, int mirror_neg, double g, double h, int nT,
                                   const double *T_dev, double *E_dev, double *C_dev, double *chi_dev,
                                   double *mag_dev, void *stream)
{
    if (n_sectors < 1 || n_sectors > FTLM_MAX_SECTORS) return fail(FTLM_EINVAL, "n_sectors out of range");
    if (R < 1 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "R or M out of range");
    if ((int64_t)n_sectors * R * M > (1ll << 31) - 1) return fail(FTLM_EUNSUPPORTED, "too many Ritz pairs");
    if (nT < 0) return fail(FTLM_EINVAL, "nT < 0");
    if (!two_sz || !dims || !theta || !weight || !m_eff) return fail(FTLM_EINVAL, "NULL host array");
    if (nT > 0 && (!T_dev || !E_dev || !C_dev || !chi_dev)) return fail(FTLM_EINVAL, "NULL device output");
    ThermoArgs a{};
    a.ns = n_sectors;
    a.R = R;
    a.M = M;
    a.mirror = mirror_neg != 0;
    a.g = g;
    a.h = h;
    for (int s = 0; s < n_sectors; ++s) {
        if (!theta[s] || !weight[s] || !m_eff[s]) return fail(FTLM_EINVAL, "NULL sector pointer");
        if (dims[s] == 0) return fail(FTLM_EINVAL, "zero sector dimension");
        a.theta[s] = theta[s];
        a.weight[s] = weight[s];
        a.meff[s] = m_eff[s];
        a.wscale[s] = (double)dims[s] / R;
        a.sz[s] = two_sz[s] / 2.0;
    }
    if (nT == 0) return FTLM_OK;
    thermo_kernel<<<nT, kThermoThreads, 0, (cudaStream_t)stream>>>(a, T_dev, E_dev, C_dev, chi_dev, mag_dev,
                                                                    nullptr, nullptr);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_partition(int n_sectors, const int *two_sz, const uint64_t *dims, int R, int M,
                                      const double *const *theta, const double *const *weight,
                                      const int *const *m_eff, int mirror_neg, double h, int nT, const double *T_dev,
                                      double *Z_dev, double *E0_dev, void *stream)
{
    if (n_sectors < 1 || n_sectors > FTLM_MAX_SECTORS) return fail(FTLM_EINVAL, "n_sectors out of range");
    if (R < 1 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "R or M out of range");
    if ((int64_t)n_sectors * R * M > (1ll << 31) - 1) return fail(FTLM_EUNSUPPORTED, "too many Ritz pairs");
    if (nT < 0) return fail(FTLM_EINVAL, "nT < 0");
    if (!two_sz || !dims || !theta || !weight || !m_eff) return fail(FTLM_EINVAL, "NULL host array");
    if (nT > 0 && (!T_dev || !Z_dev)) return fail(FTLM_EINVAL, "NULL device output");
    ThermoArgs a{};
    a.ns = n_sectors;
    a.R = R;
    a.M = M;
    a.mirror = mirror_neg != 0;
    a.g = 0.0;
    a.h = h;
    for (int s = 0; s < n_sectors; ++s) {
        if (!theta[s] || !weight[s] || !m_eff[s]) return fail(FTLM_EINVAL, "NULL sector pointer");
        if (dims[s] == 0) return fail(FTLM_EINVAL, "zero sector dimension");
        a.theta[s] = theta[s];
        a.weight[s] = weight[s];
        a.meff[s] = m_eff[s];
        a.wscale[s] = (double)dims[s] / R;
        a.sz[s] = two_sz[s] / 2.0;
    }
    if (nT == 0) return FTLM_OK;
    thermo_kernel<<<nT, kThermoThreads, 0, (cudaStream_t)stream>>>(a, T_dev, nullptr, nullptr, nullptr, nullptr,
                                                                    Z_dev, E0_dev);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}
