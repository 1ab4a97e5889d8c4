// Lanczos chains (steps a2, a4, a5): start vectors, the vector update, the Ritz
// step, and the launch sequence of ftlm_lanczos / ftlm_lanczos_from.
//
// Recurrence (Sec. 2, FTLM paragraph; Paige's ordering, no reorthogonalization):
//     y = H q_j - beta_{j-1} q_{j-1};  alpha_j = <q_j, y>;  w = y - alpha_j q_j;
//     beta_j = ||w||;  q_{j+1} = w / beta_j.
// Only two vectors per chain are stored.  The H.v launch (hv.cu) reads u_j and
// overwrites u_{j-1} with y; the update launch below overwrites y with w in place
// and publishes beta_j.  The division by beta_j is folded into the next H.v (the
// stored vectors stay un-normalized, q_j = u_j / s_j), so every step streams each
// vector exactly once per launch.  All scalars stay on the device; the host only
// queues 2 launches per step, and a chain that breaks down (beta_j <= tau) turns
// the rest of its launches into no-ops.
#include <cmath>
#include <mutex>
#include <vector>

#include "ftlm_internal.cuh"
#include "reduce.cuh"

namespace ftlm {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t chain_key(uint64_t seed, int N, int K, uint32_t r)
{
    const uint64_t tag = ((uint64_t)N << 48) | ((uint64_t)K << 32) | (uint64_t)r;
    return sm64_mix(sm64_mix(seed + kGamma) + tag + kGamma);
}

__device__ __forceinline__ double start_value(uint64_t key, uint64_t t, int dist)
{
    if (dist == FTLM_VEC_RADEMACHER) {
        const uint64_t u = sm64_mix(key + (t + 1) * kGamma);
        return (u >> 63) ? -1.0 : 1.0;
    }
    const uint64_t u1 = sm64_mix(key + (2 * t + 1) * kGamma);
    const uint64_t u2 = sm64_mix(key + (2 * t + 2) * kGamma);
    const double U1 = ((double)(u1 >> 11) + 1.0) * 0x1p-53;
    const double U2 = (double)(u2 >> 11) * 0x1p-53;
    const double two_pi = 2.0 * 3.14159265358979323846;
    return sqrt(-2.0 * log(U1)) * cos(two_pi * U2);
}

// u = start vector (generated, or copied from src), and s_1 = ||u|| of the stored
// (dtype-rounded) entries.
template <typename V>
__global__ void __launch_bounds__(kRowThreads)
start_kernel(uint32_t D, uint64_t key, int dist, const double *__restrict__ src, V *__restrict__ u,
             ChainState *st, double *partials)
{
    double part = 0.0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < D; t += stride) {
        const double v = src ? src[t] : start_value(key, t, dist);
        const V vv = (V)v;
        u[t] = vv;
        part += (double)vv * (double)vv;
    }
    part = block_sum<kRowThreads>(part);
    if (publish_partial(part, partials, &st->counter) && threadIdx.x < 32) {
        const double nrm = sqrt(total_of_partials(partials, gridDim.x));
        if (threadIdx.x == 0) {
            st->s_cur = nrm;
            st->s_prev = 1.0;
            st->beta_prev = 0.0;
            st->alpha = 0.0;
            st->m_eff = 0;
            st->stopped = (nrm > 0.0 && isfinite(nrm)) ? 0 : 1;
            st->counter = 0;
        }
    }
}

template <typename V> struct Vec2;
template <> struct Vec2<float> { using T = float4; static constexpr int n = 4; };
template <> struct Vec2<double> { using T = double2; static constexpr int n = 2; };

__device__ __forceinline__ float4 upd(float4 y, float4 u, float a, double &part)
{
    float4 w;
    w.x = fmaf(-a, u.x, y.x);
    w.y = fmaf(-a, u.y, y.y);
    w.z = fmaf(-a, u.z, y.z);
    w.w = fmaf(-a, u.w, y.w);
    part += (double)w.x * w.x + (double)w.y * w.y + ((double)w.z * w.z + (double)w.w * w.w);
    return w;
}
__device__ __forceinline__ double2 upd(double2 y, double2 u, double a, double &part)
{
    double2 w;
    w.x = fma(-a, u.x, y.x);
    w.y = fma(-a, u.y, y.y);
    part += w.x * w.x + w.y * w.y;
    return w;
}

// w = y - alpha_j q_j (in place over y), beta_j = ||w||, breakdown test.
template <typename V>
__global__ void __launch_bounds__(kRowThreads)
update_kernel(uint32_t D, V *__restrict__ y, const V *__restrict__ u, ChainState *st,
              double *partials, int j, int m_max, double tau, double *beta_row)
{
    if (st->stopped) return;
    const V a = (V)(st->alpha / st->s_cur);
    using VT = typename Vec2<V>::T;
    constexpr int W = Vec2<V>::n;
    double part = 0.0;
    const uint32_t nvec = D / W;
    const uint32_t stride = gridDim.x * blockDim.x;
    VT *yv = reinterpret_cast<VT *>(y);
    const VT *uv = reinterpret_cast<const VT *>(u);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride)
        __stcs(yv + i, upd(__ldcs(yv + i), __ldcs(uv + i), a, part));
    for (uint32_t t = nvec * W + blockIdx.x * blockDim.x + threadIdx.x; t < D; t += stride) {
        const V w = fma(-a, u[t], y[t]);
        y[t] = w;
        part += (double)w * (double)w;
    }
    part = block_sum<kRowThreads>(part);
    if (publish_partial(part, partials, &st->counter) && threadIdx.x < 32) {
        const double beta = sqrt(total_of_partials(partials, gridDim.x));
        if (threadIdx.x == 0) {
            if (j < m_max) {
                if (beta <= tau) {
                    st->stopped = 1;
                    st->m_eff = j;
                } else {
                    beta_row[j - 1] = beta;
                    st->s_prev = st->s_cur;
                    st->s_cur = beta;
                    st->beta_prev = beta;
                }
            } else {
                st->m_eff = m_max;
            }
            st->counter = 0;
        }
    }
}

__global__ void copy_meff_kernel(const ChainState *st, int *dst) { *dst = st->m_eff; }

// ---- Ritz step (a5) ---------------------------------------------------------
// Implicit symmetric tridiagonal QR with Wilkinson shift (Golub & Van Loan,
// "Matrix Computations", Sec. 8.3), deflating from the bottom.  Only the first
// row z of the accumulated rotation matrix is kept: the eigenvector matrix of T is
// the product of the rotations, so its first row gives s_{k,1}.
__device__ void givens(double a, double b, double &c, double &s)
{
    // [c s; -s c]^T [a; b] = [r; 0]
    if (b == 0.0) {
        c = 1.0;
        s = 0.0;
    } else if (fabs(b) > fabs(a)) {
        const double tau = -a / b;
        s = 1.0 / sqrt(1.0 + tau * tau);
        c = s * tau;
    } else {
        const double tau = -b / a;
        c = 1.0 / sqrt(1.0 + tau * tau);
        s = c * tau;
    }
}

__device__ bool negligible(double e, double d0, double d1)
{
    return fabs(e) <= 0x1p-52 * (fabs(d0) + fabs(d1)) || fabs(e) < 1e-290;
}

__device__ void tridiag_qr(double *d, double *e, double *z, int n)
{
    int hi = n - 1;
    const int max_sweeps = 64 * n;
    for (int sweep = 0; hi > 0 && sweep < max_sweeps;) {
        if (negligible(e[hi - 1], d[hi - 1], d[hi])) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !negligible(e[lo - 1], d[lo - 1], d[lo])) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        ++sweep;
        const double dd = 0.5 * (d[hi - 1] - d[hi]);
        const double bb = e[hi - 1];
        const double den = dd + (dd >= 0.0 ? 1.0 : -1.0) * hypot(dd, bb);
        const double mu = d[hi] - bb * (bb / den);
        double x = d[lo] - mu, zz = e[lo];
        for (int k = lo; k < hi; ++k) {
            double c, s;
            givens(x, zz, c, s);
            if (k > lo) e[k - 1] = c * x - s * zz;
            const double a = d[k], b = e[k], cc = d[k + 1];
            const double c2 = c * c, s2 = s * s, cs = c * s;
            d[k] = c2 * a - 2.0 * cs * b + s2 * cc;
            d[k + 1] = s2 * a + 2.0 * cs * b + c2 * cc;
            e[k] = cs * (a - cc) + (c2 - s2) * b;
            if (k < hi - 1) {
                x = e[k];
                zz = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            const double z0 = z[k], z1 = z[k + 1];
            z[k] = c * z0 - s * z1;
            z[k + 1] = s * z0 + c * z1;
        }
    }
}

__global__ void ritz_kernel(int M, const double *__restrict__ alpha, const double *__restrict__ beta,
                            const int *__restrict__ mv, double *theta, double *weight)
{
    extern __shared__ double sh[];
    double *d = sh, *e = sh + M, *z = sh + 2 * M;
    const int c = blockIdx.x;
    int m = mv[c];
    m = m < 0 ? 0 : (m > M ? M : m);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        d[i] = i < m ? alpha[(size_t)c * M + i] : 0.0;
        e[i] = i + 1 < m ? beta[(size_t)c * M + i] : 0.0;
        z[i] = i == 0 ? 1.0 : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0 && m > 1) {
        tridiag_qr(d, e, z, m);
        for (int i = 1; i < m; ++i) {  // ascending theta
            const double dk = d[i], zk = z[i];
            int k = i - 1;
            while (k >= 0 && d[k] > dk) {
                d[k + 1] = d[k];
                z[k + 1] = z[k];
                --k;
            }
            d[k + 1] = dk;
            z[k + 1] = zk;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        theta[(size_t)c * M + i] = i < m ? d[i] : 0.0;
        weight[(size_t)c * M + i] = i < m ? z[i] * z[i] : 0.0;
    }
}

ftlm_status launch_ritz(int n, int M, const double *alpha, const double *beta, const int *mv,
                        double *theta, double *weight, cudaStream_t stream)
{
    if (n == 0) return FTLM_OK;
    ritz_kernel<<<n, 32, 3 * (size_t)M * sizeof(double), stream>>>(M, alpha, beta, mv, theta, weight);
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

// ---- workspace -------------------------------------------------------------
uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

struct Layout {
    uint64_t vec0, vec1, partials, state, alpha, beta, meff, total;
};

Layout layout(const ftlm_basis *b, int R, int M, ftlm_dtype dtype)
{
    Layout l;
    const uint64_t vb = align256(b->D * (dtype == FTLM_F32 ? 4ull : 8ull));
    l.vec0 = 0;
    l.vec1 = vb;
    l.partials = 2 * vb;
    l.state = l.partials + align256((uint64_t)max_row_grid(b) * sizeof(double));
    l.alpha = l.state + align256(sizeof(ChainState));
    l.beta = l.alpha + align256((uint64_t)R * M * sizeof(double));
    l.meff = l.beta + align256((uint64_t)R * M * sizeof(double));
    l.total = l.meff + align256((uint64_t)R * sizeof(int));
    return l;
}

template <typename V>
int occupancy_of(const void *kern)
{
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRowThreads, 0);
    return occ;
}

template <typename V>
ftlm_status run_chains(const ftlm_basis *b, int R, int M, uint64_t seed, int dist, const double *src,
                       ftlm_dtype dtype, char *ws, const Layout &lay, double *theta, double *weight,
                       int *m_eff, double *alpha_dev, double *beta_dev, cudaStream_t stream)
{
    static int occ_start = -1, occ_upd = -1;
    if (occ_start < 0) occ_start = occupancy_of<V>((const void *)start_kernel<V>);
    if (occ_upd < 0) occ_upd = occupancy_of<V>((const void *)update_kernel<V>);
    V *vec[2] = {(V *)(ws + lay.vec0), (V *)(ws + lay.vec1)};
    double *partials = (double *)(ws + lay.partials);
    ChainState *st = (ChainState *)(ws + lay.state);
    double *alpha_ws = (double *)(ws + lay.alpha);
    double *beta_ws = (double *)(ws + lay.beta);
    int *meff_ws = (int *)(ws + lay.meff);
    const uint32_t D = (uint32_t)b->D;
    const int m_max = (uint64_t)M < b->D ? M : (int)b->D;
    const double tau = dtype == FTLM_F32 ? b->tau32 : b->tau64;
    const int g_start = row_grid(b, D, occ_start);
    const int g_upd = row_grid(b, (D + Vec2<V>::n - 1) / Vec2<V>::n, occ_upd);

    FTLM_CUDA(cudaMemsetAsync(st, 0, sizeof(ChainState), stream));
    FTLM_CUDA(cudaMemsetAsync(alpha_ws, 0, (size_t)R * M * sizeof(double), stream));
    FTLM_CUDA(cudaMemsetAsync(beta_ws, 0, (size_t)R * M * sizeof(double), stream));
    for (int r = 0; r < R; ++r) {
        const uint64_t key = chain_key(seed, b->N, b->K, (uint32_t)r);
        start_kernel<V><<<g_start, kRowThreads, 0, stream>>>(D, key, dist, src ? src + (size_t)r * D : nullptr,
                                                             vec[0], st, partials);
        FTLM_CUDA(cudaGetLastError());
        int cur = 0;
        for (int j = 1; j <= m_max; ++j) {
            LanczosHv epi{vec[1 - cur], st, partials, alpha_ws + (size_t)r * M + (j - 1), j};
            ftlm_status s = launch_hv(b, dtype, vec[cur], vec[1 - cur], &epi, stream);
            if (s != FTLM_OK) return s;
            void *tok = profile_begin(kProfUpdate, stream);
            update_kernel<V><<<g_upd, kRowThreads, 0, stream>>>(D, vec[1 - cur], vec[cur], st, partials, j,
                                                                m_max, tau, beta_ws + (size_t)r * M);
            profile_end(tok, stream);
            FTLM_CUDA(cudaGetLastError());
            cur = 1 - cur;
        }
        copy_meff_kernel<<<1, 1, 0, stream>>>(st, meff_ws + r);
        FTLM_CUDA(cudaGetLastError());
    }
    ftlm_status s = launch_ritz(R, M, alpha_ws, beta_ws, meff_ws, theta, weight, stream);
    if (s != FTLM_OK) return s;
    FTLM_CUDA(cudaMemcpyAsync(m_eff, meff_ws, (size_t)R * sizeof(int), cudaMemcpyDeviceToDevice, stream));
    if (alpha_dev)
        FTLM_CUDA(cudaMemcpyAsync(alpha_dev, alpha_ws, (size_t)R * M * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    if (beta_dev)
        FTLM_CUDA(cudaMemcpyAsync(beta_dev, beta_ws, (size_t)R * M * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    return FTLM_OK;
}

ftlm_status lanczos_common(const ftlm_basis *b, int R, int M, uint64_t seed, int dist, const double *src,
                           ftlm_dtype dtype, void *work, uint64_t work_bytes, double *theta,
                           double *weight, int *m_eff, double *alpha_dev, double *beta_dev, void *stream)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (R < 1) return fail(FTLM_EINVAL, "R < 1");
    if (M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "M out of range");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    if (dist != FTLM_VEC_GAUSS && dist != FTLM_VEC_RADEMACHER) return fail(FTLM_EINVAL, "bad distribution");
    if (!theta || !weight || !m_eff) return fail(FTLM_EINVAL, "NULL output");
    if (!work || ((uintptr_t)work & 255u)) return fail(FTLM_EINVAL, "workspace NULL or not 256-byte aligned");
    const Layout lay = layout(b, R, M, dtype);
    if (work_bytes < lay.total) return fail(FTLM_ENOMEM, "workspace smaller than ftlm_lanczos_workspace_bytes()");
    return dtype == FTLM_F32
               ? run_chains<float>(b, R, M, seed, dist, src, dtype, (char *)work, lay, theta, weight, m_eff,
                                   alpha_dev, beta_dev, (cudaStream_t)stream)
               : run_chains<double>(b, R, M, seed, dist, src, dtype, (char *)work, lay, theta, weight, m_eff,
                                    alpha_dev, beta_dev, (cudaStream_t)stream);
}

// Scratch of ftlm_lanczos_noalloc, for callers that cannot allocate device memory.
// Host code sees only a host-side stand-in for this symbol; its device address is
// looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FTLM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on first use).
ftlm_status noalloc_scratch(void **out)
{
    int dev = 0;
    FTLM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(FTLM_EUNSUPPORTED, "device index beyond 64");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        FTLM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FTLM_OK;
}

}  // namespace

}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_lanczos_noalloc(const ftlm_basis *b, int R, int M, uint64_t seed,
                                            ftlm_vec_dist dist, ftlm_dtype dtype, double *theta_dev,
                                            double *weight_dev, int *m_eff_dev, double *alpha_dev,
                                            double *beta_dev, void *stream)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (R < 1 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "R or M out of range");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    const uint64_t need = layout(b, R, M, dtype).total;
    if (need > FTLM_NOALLOC_SCRATCH_BYTES)
        return fail(FTLM_EUNSUPPORTED, "workspace of " + std::to_string(need) +
                                           " bytes exceeds the static scratch of FTLM_NOALLOC_SCRATCH_BYTES (" +
                                           std::to_string(FTLM_NOALLOC_SCRATCH_BYTES) + " bytes)");
    void *scratch = nullptr;
    ftlm_status s = noalloc_scratch(&scratch);
    if (s != FTLM_OK) return s;
    return lanczos_common(b, R, M, seed, dist, nullptr, dtype, scratch, FTLM_NOALLOC_SCRATCH_BYTES,
                          theta_dev, weight_dev, m_eff_dev, alpha_dev, beta_dev, stream);
}

extern "C" ftlm_status ftlm_lanczos_workspace_bytes(const ftlm_basis *b, int R, int M, ftlm_dtype dtype,
                                                    uint64_t *bytes)
{
    if (!b || !bytes) return fail(FTLM_EINVAL, "NULL argument");
    if (R < 1 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "R or M out of range");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    *bytes = layout(b, R, M, dtype).total;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_lanczos(const ftlm_basis *b, int R, int M, uint64_t seed, ftlm_vec_dist dist,
                                    ftlm_dtype dtype, void *work_dev, uint64_t work_bytes, double *theta_dev,
                                    double *weight_dev, int *m_eff_dev, double *alpha_dev, double *beta_dev,
                                    void *stream)
{
    return lanczos_common(b, R, M, seed, dist, nullptr, dtype, work_dev, work_bytes, theta_dev, weight_dev,
                          m_eff_dev, alpha_dev, beta_dev, stream);
}

extern "C" ftlm_status ftlm_lanczos_from(const ftlm_basis *b, int R, int M, const double *start_dev,
                                         ftlm_dtype dtype, void *work_dev, uint64_t work_bytes,
                                         double *theta_dev, double *weight_dev, int *m_eff_dev,
                                         double *alpha_dev, double *beta_dev, void *stream)
{
    if (!start_dev) return fail(FTLM_EINVAL, "start_dev is NULL");
    return lanczos_common(b, R, M, 0, FTLM_VEC_GAUSS, start_dev, dtype, work_dev, work_bytes, theta_dev,
                          weight_dev, m_eff_dev, alpha_dev, beta_dev, stream);
}

extern "C" ftlm_status ftlm_ritz(int n, int M, const double *alpha_dev, const double *beta_dev,
                                 const int *m_dev, double *theta_dev, double *weight_dev, void *stream)
{
    if (n < 0 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "n or M out of range");
    if (n > 0 && (!alpha_dev || !beta_dev || !m_dev || !theta_dev || !weight_dev))
        return fail(FTLM_EINVAL, "NULL device pointer");
    return launch_ritz(n, M, alpha_dev, beta_dev, m_dev, theta_dev, weight_dev, (cudaStream_t)stream);
}
