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
// queues 2 launches per step (3 for CR sectors, whose H.v launch leaves alpha_j
// as per-tile sums for a short second launch), and a chain that breaks down
// (beta_j <= tau) turns the rest of its launches into no-ops.
#include <cmath>
#include <cstdlib>
#include <atomic>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "vec.cuh"
#include "rng.cuh"
#include "tridiag.cuh"

namespace ftlm {

namespace {

struct Keys {
    uint64_t k[kMaxBlock];
};

// Finish a launch's per-chain reduction: every block stores its B partial sums;
// the last block to arrive returns true (in every thread) and the caller's warp 0
// adds the partials of chain r in block order with chain_total().
template <int B>
__device__ __forceinline__ bool publish_partials(const double (&part)[B], double *partials, unsigned int *counter)
{
    __shared__ double s_part[B];
    __shared__ bool s_last;
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const double v = block_sum<kRowThreads>(part[r]);
        if (threadIdx.x == 0) s_part[r] = v;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < B; ++r) partials[(size_t)blockIdx.x * B + r] = s_part[r];
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return s_last;
}

// Fixed-order total of chain r's partials; call from warp 0, valid in lane 0.
template <int B>
__device__ __forceinline__ double chain_total(const double *partials, int r)
{
    double v = 0.0;
    for (int g = threadIdx.x; g < (int)gridDim.x; g += 32) v += __ldcg(partials + (size_t)g * B + r);
    return warp_sum(v);
}

// Start vectors of a block of B chains (generated, or copied from src rows of
// length D), interleaved, and s_1 = ||u|| of each chain's stored (dtype-rounded)
// entries.
template <typename V, int B>
__global__ void __launch_bounds__(kRowThreads)
start_kernel(uint32_t D, const Keys keys, int dist, const double *__restrict__ src, V *__restrict__ u,
             ChainState *st, double *partials, unsigned int *counter)
{
    DotAcc<V> acc[B];
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < D; t += stride) {
        V out[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            const double v = src ? src[(size_t)r * D + t] : start_value(keys.k[r], t, dist);
            out[r] = (V)v;
            acc[r].add(out[r], out[r]);
        }
        st_vec<B>(u + (size_t)t * B, out);
    }
    double part[B];
#pragma unroll
    for (int r = 0; r < B; ++r) part[r] = acc[r].value();
    if (publish_partials<B>(part, partials, counter) && threadIdx.x < 32) {
        for (int r = 0; r < B; ++r) {
            const double nrm = sqrt(chain_total<B>(partials, r));
            if (threadIdx.x == 0) {
                ChainState &c = st[r];
                c.s_cur = nrm;
                c.s_prev = 1.0;
                c.beta_prev = 0.0;
                c.alpha = 0.0;
                c.m_eff = 0;
                c.stopped = (nrm > 0.0 && isfinite(nrm)) ? 0 : 1;
            }
        }
        if (threadIdx.x == 0) *counter = 0;
    }
}

// w = y - alpha_j q_j per chain (in place over y), beta_j = ||w||, breakdown test.
// Columns of chains that have ended are set to zero.  The block is processed in
// units of U = max(B, 16 bytes) values; entry e of a unit belongs to chain e % B.
template <typename V, int B>
__global__ void __launch_bounds__(kRowThreads)
update_kernel(uint32_t D, V *__restrict__ y, const V *__restrict__ u, ChainState *st, double *partials,
              unsigned int *counter, int j, int m_max, double tau, double *beta_out, int beta_stride)
{
    V a[B];
    bool zero[B];
    bool all_stopped = true;
#pragma unroll
    for (int r = 0; r < B; ++r) {
        zero[r] = st[r].stopped != 0;
        all_stopped &= zero[r];
        a[r] = zero[r] ? (V)0 : (V)(st[r].alpha / st[r].s_cur);
    }
    if (all_stopped) return;
    constexpr int W = 16 / (int)sizeof(V);
    constexpr int U = B > W ? B : W;
    DotAcc<V> acc[B];
    const uint64_t total = (uint64_t)D * B, units = total / U;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < units; i += stride) {
        V yv[U], uv[U], w[U];
        ld_vec<U>(y + i * U, yv, true);
        ld_vec<U>(u + i * U, uv, true);
#pragma unroll
        for (int e = 0; e < U; ++e) {
            const int r = e % B;
            w[e] = zero[r] ? (V)0 : fma(-a[r], uv[e], yv[e]);
            acc[r].add(w[e], w[e]);
        }
        st_vec<U>(y + i * U, w);
    }
    for (uint64_t e = units * U + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
        // only reached with B = 1 (and D not a multiple of U)
        const V w = zero[0] ? (V)0 : fma(-a[0], u[e], y[e]);
        y[e] = w;
        acc[0].add(w, w);
    }
    double part[B];
#pragma unroll
    for (int r = 0; r < B; ++r) part[r] = acc[r].value();
    if (publish_partials<B>(part, partials, counter) && threadIdx.x < 32) {
        for (int r = 0; r < B; ++r) {
            const double beta = sqrt(chain_total<B>(partials, r));
            if (threadIdx.x == 0 && !st[r].stopped) {
                ChainState &c = st[r];
                if (j < m_max) {
                    if (beta <= tau) {
                        c.stopped = 1;
                        c.m_eff = j;
                    } else {
                        beta_out[(size_t)r * beta_stride + (j - 1)] = beta;
                        c.s_prev = c.s_cur;
                        c.s_cur = beta;
                        c.beta_prev = beta;
                    }
                } else {
                    c.m_eff = m_max;
                }
            }
        }
        if (threadIdx.x == 0) *counter = 0;
    }
}

__global__ void copy_meff_kernel(const ChainState *st, int B, int *dst)
{
    if (threadIdx.x < B) dst[threadIdx.x] = st[threadIdx.x].m_eff;
}

// Tridiagonal problems of this translation unit that did not converge (read and
// cleared by ftlm_ritz_status); one copy per device.
__device__ unsigned long long g_ritz_unconverged;

// One thread per chain; T chains per CTA.  A chain whose QR iteration does not
// converge within max_sweeps gets NaN Ritz values and weights.  rows == nullptr:
// chain c reads row c of alpha/beta/mv and writes row c of theta/weight; else
// rows[c] names its coefficient row and its outputs (and m_eff is copied out).
__global__ void ritz_kernel(int n, int M, const double *__restrict__ alpha, const double *__restrict__ beta,
                            const int *__restrict__ mv, double *theta, double *weight, const RitzRow *rows,
                            int max_sweeps)
{
    extern __shared__ double sh[];
    const int T = blockDim.x, i = threadIdx.x;
    const int c = blockIdx.x * T + i;
    if (c >= n) return;
    Strided d{sh + i, T}, e{sh + (size_t)M * T + i, T}, z{sh + (size_t)2 * M * T + i, T};
    size_t row;
    double *th, *wt;
    if (rows) {
        const RitzRow r = rows[c];
        row = r.row;
        th = r.theta;
        wt = r.weight;
    } else {
        row = (size_t)c;
        th = theta + row * M;
        wt = weight + row * M;
    }
    int m = mv[row];
    if (rows) rows[c].m_eff[0] = m;
    m = m < 0 ? 0 : (m > M ? M : m);
    for (int k = 0; k < m; ++k) {
        d[k] = alpha[row * M + k];
        e[k] = k + 1 < m ? beta[row * M + k] : 0.0;
        z[k] = k == 0 ? 1.0 : 0.0;
    }
    bool ok = true;
    if (m > 1) {
        ok = tridiag_qr(d, e, z, m, max_sweeps);
        if (ok) sort_ascending(d, z, m);
        else atomicAdd(&g_ritz_unconverged, 1ull);
    }
    for (int k = 0; k < M; ++k) {
        th[k] = k < m ? (ok ? d[k] : NAN) : 0.0;
        wt[k] = k < m ? (ok ? z[k] * z[k] : NAN) : 0.0;
    }
}

}  // namespace

std::atomic<int> g_ritz_max_sweeps{0};
int ritz_max_sweeps() { return g_ritz_max_sweeps.load(std::memory_order_relaxed); }

namespace {

ftlm_status ritz_launch(int n, int M, const double *alpha, const double *beta, const int *mv, double *theta,
                        double *weight, const RitzRow *rows, cudaStream_t stream)
{
    if (n == 0) return FTLM_OK;
    constexpr size_t kSmemMax = 96 * 1024;
    int occ = 1;
    FTLM_CUDA(kernel_occupancy((const void *)ritz_kernel, 32, kSmemMax, true, &occ));
    const size_t per_chain = 3 * (size_t)M * sizeof(double);
    int T = (int)(kSmemMax / per_chain);
    T = T < 1 ? 1 : (T > 32 ? 32 : T);
    if (T > n) T = n;
    const int grid = (n + T - 1) / T;
    ritz_kernel<<<grid, T, per_chain * T, stream>>>(n, M, alpha, beta, mv, theta, weight, rows, ritz_max_sweeps());
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

}  // namespace

ftlm_status launch_ritz(int n, int M, const double *alpha, const double *beta, const int *mv,
                        double *theta, double *weight, cudaStream_t stream)
{
    return ritz_launch(n, M, alpha, beta, mv, theta, weight, nullptr, stream);
}

ftlm_status launch_ritz_rows(int n, int M, const double *alpha, const double *beta, const int *mv,
                             const RitzRow *rows, cudaStream_t stream)
{
    return ritz_launch(n, M, alpha, beta, mv, nullptr, nullptr, rows, stream);
}

namespace {

// ---- workspace and block plan -------------------------------------------
uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

// Widest block of chains: the width set by ftlm_lanczos_set_block, else FTLM_BLOCK
// (1, 4, 8 or 16), else 8 vectors (FP32) or 4 (FP64).
std::atomic<int> g_block_width{0};

int max_block(ftlm_dtype dtype)
{
    static const int over = [] {
        const char *e = getenv("FTLM_BLOCK");
        const int v = e ? atoi(e) : 0;
        return valid_block(v) ? v : 0;
    }();
    const int set = g_block_width.load(std::memory_order_relaxed);
    if (set) return set;
    return over ? over : (dtype == FTLM_F32 ? 8 : 4);
}

// Split R chains into blocks: the widest allowed width in {16, 8, 4} that fits the
// chains left, then single chains for fewer than 4.  bmax = 0: max_block(dtype).
std::vector<int> block_plan(int R, ftlm_dtype dtype, int bmax)
{
    if (!bmax) bmax = max_block(dtype);
    std::vector<int> plan;
    int left = R;
    for (int w : {16, 8, 4}) {
        if (w > bmax) continue;
        while (left >= w) {
            plan.push_back(w);
            left -= w;
        }
    }
    while (left-- > 0) plan.push_back(1);
    return plan;
}

struct Layout {
    int bw;  // widest block
    uint64_t vec0, vec1, partials, state, alpha, beta, meff, tiles, total;
};

Layout layout(const ftlm_basis *b, int R, int M, ftlm_dtype dtype, int bmax = 0)
{
    Layout l;
    l.bw = 1;
    for (int w : block_plan(R, dtype, bmax)) l.bw = w > l.bw ? w : l.bw;
    const uint64_t vb = align256(b->D * (uint64_t)l.bw * (dtype == FTLM_F32 ? 4ull : 8ull));
    l.vec0 = 0;
    l.vec1 = vb;
    l.partials = 2 * vb;
    l.state = l.partials + align256((uint64_t)max_row_grid(b) * l.bw * sizeof(double));
    l.alpha = l.state + align256(l.bw * sizeof(ChainState) + 64);
    l.beta = l.alpha + align256((uint64_t)R * M * sizeof(double));
    l.meff = l.beta + align256((uint64_t)R * M * sizeof(double));
    l.tiles = l.meff + align256((uint64_t)R * sizeof(int));
    // per-tile alpha sums of dynamically ordered H.v launches (B >= 4 has the most tiles)
    l.total = l.tiles + align256((uint64_t)hv_lanczos_tiles(b, 4) * l.bw * sizeof(double));
    return l;
}

// One block of B chains: start vectors, then min(M, D) fused H.v + update launches.
template <typename V, int B>
ftlm_status run_block(const ftlm_basis *b, int M, int r0, int chain0, uint64_t seed, int dist, const double *src,
                      ftlm_dtype dtype, char *ws, const Layout &lay, cudaStream_t stream)
{
    int occ_start = 1, occ_upd = 1;
    FTLM_CUDA(kernel_occupancy((const void *)start_kernel<V, B>, kRowThreads, 0, false, &occ_start));
    FTLM_CUDA(kernel_occupancy((const void *)update_kernel<V, B>, kRowThreads, 0, false, &occ_upd));
    V *vec[2] = {(V *)(ws + lay.vec0), (V *)(ws + lay.vec1)};
    double *partials = (double *)(ws + lay.partials);
    ChainState *st = (ChainState *)(ws + lay.state);
    unsigned int *counter = (unsigned int *)(st + lay.bw);
    double *alpha_ws = (double *)(ws + lay.alpha);
    double *beta_ws = (double *)(ws + lay.beta);
    int *meff_ws = (int *)(ws + lay.meff);
    const uint32_t D = (uint32_t)b->D;
    const int m_max = (uint64_t)M < b->D ? M : (int)b->D;
    const double tau = dtype == FTLM_F32 ? b->tau32 : b->tau64;
    constexpr int W = 16 / (int)sizeof(V);
    constexpr int U = B > W ? B : W;
    const int g_start = row_grid(b, D, occ_start);
    const int g_upd = row_grid(b, ((uint64_t)D * B + U - 1) / U, occ_upd);

    FTLM_CUDA(cudaMemsetAsync(st, 0, lay.bw * sizeof(ChainState) + 64, stream));
    Keys keys{};
    for (int r = 0; r < B; ++r) keys.k[r] = chain_key(seed, b->key_n, b->K, (uint32_t)(chain0 + r0 + r));
    start_kernel<V, B><<<g_start, kRowThreads, 0, stream>>>(D, keys, dist, src ? src + (size_t)r0 * D : nullptr,
                                                           vec[0], st, partials, counter);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    int cur = 0;
    for (int j = 1; j <= m_max; ++j) {
        LanczosHv epi{st, partials, counter, alpha_ws + (size_t)r0 * M + (j - 1), M, j, (double *)(ws + lay.tiles)};
        ftlm_status s = launch_hv(b, dtype, B, vec[cur], vec[1 - cur], &epi, stream);
        if (s != FTLM_OK) return s;
        void *tok = profile_begin(kProfUpdate, stream);
        update_kernel<V, B><<<g_upd, kRowThreads, 0, stream>>>(D, vec[1 - cur], vec[cur], st, partials, counter, j,
                                                               m_max, tau, beta_ws + (size_t)r0 * M, M);
        note_launch();
        profile_end(tok, stream);
        FTLM_CUDA(cudaGetLastError());
        cur = 1 - cur;
    }
    copy_meff_kernel<<<1, 32, 0, stream>>>(st, B, meff_ws + r0);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V>
ftlm_status run_chains(const ftlm_basis *b, int R, int M, int chain0, uint64_t seed, int dist, const double *src,
                       ftlm_dtype dtype, int bmax, char *ws, const Layout &lay, double *theta, double *weight,
                       int *m_eff, double *alpha_dev, double *beta_dev, cudaStream_t stream)
{
    double *alpha_ws = (double *)(ws + lay.alpha);
    double *beta_ws = (double *)(ws + lay.beta);
    int *meff_ws = (int *)(ws + lay.meff);
    FTLM_CUDA(cudaMemsetAsync(alpha_ws, 0, (size_t)R * M * sizeof(double), stream));
    FTLM_CUDA(cudaMemsetAsync(beta_ws, 0, (size_t)R * M * sizeof(double), stream));
    int r0 = 0;
    for (int B : block_plan(R, dtype, bmax)) {
        ftlm_status s;
        switch (B) {
        case 16: s = run_block<V, 16>(b, M, r0, chain0, seed, dist, src, dtype, ws, lay, stream); break;
        case 8: s = run_block<V, 8>(b, M, r0, chain0, seed, dist, src, dtype, ws, lay, stream); break;
        case 4: s = run_block<V, 4>(b, M, r0, chain0, seed, dist, src, dtype, ws, lay, stream); break;
        default: s = run_block<V, 1>(b, M, r0, chain0, seed, dist, src, dtype, ws, lay, stream); break;
        }
        if (s != FTLM_OK) return s;
        r0 += B;
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

}  // namespace

ftlm_status lanczos_run(const ftlm_basis *b, int R, int M, int chain0, uint64_t seed, int dist, const double *src,
                        ftlm_dtype dtype, void *work, uint64_t work_bytes, double *theta, double *weight,
                        int *m_eff, double *alpha_dev, double *beta_dev, cudaStream_t stream, int bmax)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (R < 1) return fail(FTLM_EINVAL, "R < 1");
    if (bmax && !valid_block(bmax)) return fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    if (!bmax) bmax = max_block(dtype);
    if (M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "M out of range");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    if (dist != FTLM_VEC_GAUSS && dist != FTLM_VEC_RADEMACHER) return fail(FTLM_EINVAL, "bad distribution");
    if (!theta || !weight || !m_eff) return fail(FTLM_EINVAL, "NULL output");
    if (!work || ((uintptr_t)work & 255u)) return fail(FTLM_EINVAL, "workspace NULL or not 256-byte aligned");
    const Layout lay = layout(b, R, M, dtype, bmax);
    if (work_bytes < lay.total) return fail(FTLM_ENOMEM, "workspace smaller than ftlm_lanczos_workspace_bytes()");
    return dtype == FTLM_F32
               ? run_chains<float>(b, R, M, chain0, seed, dist, src, dtype, bmax, (char *)work, lay, theta, weight,
                                   m_eff, alpha_dev, beta_dev, stream)
               : run_chains<double>(b, R, M, chain0, seed, dist, src, dtype, bmax, (char *)work, lay, theta, weight,
                                    m_eff, alpha_dev, beta_dev, stream);
}

uint64_t lanczos_workspace(const ftlm_basis *b, int R, int M, ftlm_dtype dtype, int bmax)
{
    return layout(b, R, M, dtype, bmax).total;
}

namespace {

// Scratch of ftlm_lanczos_noalloc, for callers that cannot allocate device memory.
// Host code sees only a host-side stand-in for this symbol; its device address is
// looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FTLM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
// Per device: the context the address was looked up in (cuCtxGetId, never reused
// within a process) and the address.  A device reset gives the device a new
// primary context, and the module with the array is loaded again at a new
// address; the id comparison makes the next call look it up again.
struct NoallocSlot {
    unsigned long long ctx_id;
    void *ptr;
};
NoallocSlot g_noalloc[kMaxDevices] = {};

// Id of the current context, from the driver through the runtime's entry-point
// query (no link-time dependency on the driver library); false if unavailable.
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch on the current device: looked up with
// cudaGetSymbolAddress on the first call in a context, cached for later calls.
// (Before any runtime call on this thread no context may be current yet; then the
// address is looked up, which binds the primary context, and cached from the
// next call on.)
ftlm_status noalloc_scratch(void **out)
{
    int dev = 0;
    FTLM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(FTLM_EUNSUPPORTED, "device index beyond 64");
    unsigned long long ctx = 0;
    const bool have_id = current_context_id(&ctx);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocSlot &slot = g_noalloc[dev];
    if (!slot.ptr || !have_id || slot.ctx_id != ctx) {
        void *p = nullptr;
        FTLM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        slot.ptr = p;
        slot.ctx_id = have_id ? ctx : 0;
    }
    *out = slot.ptr;
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
    return lanczos_run(b, R, M, 0, seed, dist, nullptr, dtype, scratch, FTLM_NOALLOC_SCRATCH_BYTES, theta_dev,
                       weight_dev, m_eff_dev, alpha_dev, beta_dev, (cudaStream_t)stream);
}

extern "C" ftlm_status ftlm_lanczos_set_block(int width)
{
    if (width != 0 && !valid_block(width)) return fail(FTLM_EINVAL, "block width must be 0, 1, 4, 8 or 16");
    g_block_width.store(width, std::memory_order_relaxed);
    return FTLM_OK;
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
    return lanczos_run(b, R, M, 0, seed, dist, nullptr, dtype, work_dev, work_bytes, theta_dev, weight_dev, m_eff_dev,
                       alpha_dev, beta_dev, (cudaStream_t)stream);
}

extern "C" ftlm_status ftlm_lanczos_from(const ftlm_basis *b, int R, int M, const double *start_dev,
                                         ftlm_dtype dtype, void *work_dev, uint64_t work_bytes,
                                         double *theta_dev, double *weight_dev, int *m_eff_dev,
                                         double *alpha_dev, double *beta_dev, void *stream)
{
    if (!start_dev) return fail(FTLM_EINVAL, "start_dev is NULL");
    return lanczos_run(b, R, M, 0, 0, FTLM_VEC_GAUSS, start_dev, dtype, work_dev, work_bytes, theta_dev, weight_dev,
                       m_eff_dev, alpha_dev, beta_dev, (cudaStream_t)stream);
}

namespace ftlm {
ftlm_status ritz_unconverged_take(cudaStream_t stream, uint64_t *count)
{
    unsigned long long v = 0, zero = 0;
    FTLM_CUDA(cudaMemcpyFromSymbolAsync(&v, g_ritz_unconverged, sizeof(v), 0, cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaMemcpyToSymbolAsync(g_ritz_unconverged, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    *count = v;
    return FTLM_OK;
}
}  // namespace ftlm

extern "C" ftlm_status ftlm_ritz_status(void *stream, uint64_t *unconverged)
{
    uint64_t a = 0, b = 0;
    ftlm_status s = ritz_unconverged_take((cudaStream_t)stream, &a);
    if (s == FTLM_OK) s = ghost_unconverged_take((cudaStream_t)stream, &b);
    if (s != FTLM_OK) return s;
    if (unconverged) *unconverged = a + b;
    if (a + b) return fail(FTLM_ENOCONV, std::to_string(a + b) + " tridiagonal eigenproblem(s) did not converge");
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_ritz_set_max_sweeps(int sweeps)
{
    if (sweeps < 0) return fail(FTLM_EINVAL, "sweeps < 0");
    g_ritz_max_sweeps.store(sweeps, std::memory_order_relaxed);
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_ritz(int n, int M, const double *alpha_dev, const double *beta_dev,
                                 const int *m_dev, double *theta_dev, double *weight_dev, void *stream)
{
    if (n < 0 || M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "n or M out of range");
    if (n > 0 && (!alpha_dev || !beta_dev || !m_dev || !theta_dev || !weight_dev))
        return fail(FTLM_EINVAL, "NULL device pointer");
    return launch_ritz(n, M, alpha_dev, beta_dev, m_dev, theta_dev, weight_dev, (cudaStream_t)stream);
}
