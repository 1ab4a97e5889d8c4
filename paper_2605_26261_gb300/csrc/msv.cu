// Lanczos chains of many sectors advanced together, one launch per step kind
// (steps a2-a4 over a set of sectors).
//
// The units are blocks of B chains of mid-sized and large sectors.  Their rows are
// cut into tiles (tile_rows, default kMsTileRows); one launch walks the tiles of every unit of a
// wave (a persistent grid; the H.v launch hands tiles out in order from a counter,
// so at any moment the GPU works on a window of consecutive tiles -- one or two
// sectors -- whose vectors stay in L2).  Per Lanczos step there are two launches for the whole wave: the fused
// H.v + alpha epilogue and the w/beta update, each with per-unit reductions:
// every tile stores its partial sums, and the CTA that finishes a unit's last tile
// (an atomic ticket per unit, no waiting) adds the unit's partials in tile order.
// A unit's arithmetic depends only on its own tiles, so its results are the same
// whatever other units share the launch, and bit-reproducible.
//
// The recurrence, stop test and chain state follow ftlm_lanczos exactly (Paige's
// ordering, 1/beta folded into the next H.v, columns of ended chains zeroed).
#include "epi.cuh"
#include "ftlm_internal.cuh"
#include "msv.cuh"
#include "reduce.cuh"
#include "rng.cuh"
#include "rows.cuh"
#include "spin_rows.cuh"
#include "vec.cuh"

namespace ftlm {

namespace {

struct UnitView {
    const MsUnit *u;
    char *ws;
    __device__ ChainState *st() const { return reinterpret_cast<ChainState *>(ws + u->off_st); }
    __device__ unsigned int *counter() const
    {
        return reinterpret_cast<unsigned int *>(ws + u->off_st + (size_t)kMaxBlock * sizeof(ChainState));
    }
    __device__ double *partials() const { return reinterpret_cast<double *>(ws + u->off_part); }
    template <typename V> __device__ V *vec(int which) const
    {
        return reinterpret_cast<V *>(ws + (which ? u->off_v1 : u->off_v0));
    }
};

// Store this tile's B block sums at tile slot k of the unit; returns true (in every
// thread) in the CTA that completes the unit.
// The B sums share three barriers: one transposed warp tree for all chains, then
// thread r adds chain r's warp sums in warp order (fixed order, reproducible).
template <typename V, int B>
__device__ __forceinline__ bool tile_publish(DotAcc<V> (&acc)[B], double *partials, uint32_t k,
                                             unsigned int *counter, uint32_t n_tiles)
{
    constexpr int kWarps = kRowThreads / 32;
    __shared__ double s_w[kWarps][B];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const DotAcc<V> t = warp_sum_multi<V, B>(acc);
    if (lane < B) s_w[wid][warp_multi_index<B>(lane)] = t.value();
    __syncthreads();
    if (threadIdx.x < B) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < kWarps; ++i) t += s_w[i][threadIdx.x];
        partials[(size_t)k * B + threadIdx.x] = t;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == n_tiles - 1;
    __syncthreads();
    return s_last;
}

// Fixed-order total of chain r over the unit's tiles; warp 0, valid in lane 0.
template <int B>
__device__ __forceinline__ double tile_total(const double *partials, uint32_t n_tiles, int r)
{
    double v = 0.0;
    for (uint32_t k = threadIdx.x; k < n_tiles; k += 32) v += __ldcg(partials + (size_t)k * B + r);
    return warp_sum(v);
}

// Start vectors of the units with j0 == jstart (every unit of a batch: jstart = 0).
template <typename V, int B>
__global__ void __launch_bounds__(kRowThreads)
ms_start_kernel(const MsUnit *__restrict__ units, const uint32_t *__restrict__ tile_unit, uint32_t n_tiles, int dist,
                char *ws, int jstart)
{
    for (uint32_t g = blockIdx.x; g < n_tiles; g += gridDim.x) {
        const UnitView uv{units + tile_unit[g], ws};
        const MsUnit &U = *uv.u;
        if (U.j0 != jstart) continue;  // CTA-uniform
        const uint32_t k = g - U.stile0, D = U.s.D;
        uint64_t key[B];
#pragma unroll
        for (int r = 0; r < B; ++r) key[r] = chain_key(U.seed, U.key_n, U.K, (uint32_t)(U.chain0 + r));
        V *u0 = uv.vec<V>(0);
        DotAcc<V> acc[B];
        const uint32_t row1 = min(D, (k + 1) * U.stream_rows);
        for (uint32_t t = k * U.stream_rows + threadIdx.x; t < row1; t += kRowThreads) {
            V out[B];
#pragma unroll
            for (int r = 0; r < B; ++r) {
                out[r] = r < U.nact ? (V)start_value(key[r], t, dist) : (V)0;
                acc[r].add(out[r], out[r]);
            }
            st_vec<B>(u0 + (size_t)t * B, out);
        }
        if (tile_publish<V, B>(acc, uv.partials(), k, uv.counter(), U.n_stiles) && threadIdx.x < 32) {
            ChainState *st = uv.st();
            for (int r = 0; r < B; ++r) {
                const double nrm = sqrt(tile_total<B>(uv.partials(), U.n_stiles, r));
                if (threadIdx.x == 0) {
                    ChainState &c = st[r];
                    c.s_cur = nrm;
                    c.s_prev = 1.0;
                    c.beta_prev = 0.0;
                    c.alpha = 0.0;
                    c.m_eff = 0;
                    c.stopped = (r < U.nact && nrm > 0.0 && isfinite(nrm)) ? 0 : 1;
                }
            }
            if (threadIdx.x == 0) *uv.counter() = 0;
        }
        __syncthreads();
    }
}

// Step j: y = H q_j - beta_{j-1} q_{j-1} over the u_{j-1} block and alpha_j, for
// every tile of every unit (x = u_j is block (j - 1) % 2, y block j % 2).
// Resident CTAs per SM the registers are cut for: FP32 blocks up to 8 fit 3 CTAs
// without spills (FP64 blocks of 4 and 8 need 2), single vectors 4 (3 for FP64
// general-spin rows).
template <typename V, int B, int KIND> __host__ __device__ constexpr int ms_min_ctas()
{
    return B >= 16 ? 1
                   : (sizeof(V) == 8 && B >= 4 ? 2 : (B >= 4 ? 3 : (sizeof(V) == 8 && KIND == kMsSpin ? 3 : 4)));
}

template <typename V, int KIND, int B, int C>
__global__ void __launch_bounds__(kRowThreads, ms_min_ctas<V, B, KIND>())
ms_hv_kernel(const MsUnit *__restrict__ units, const uint32_t *__restrict__ tile_unit, uint32_t n_tiles, int j,
             int M, double *alpha, char *ws)
{
    constexpr bool CLT = KIND == kMsClt, SPIN = KIND == kMsSpin;
    extern __shared__ uint16_t s_tlo[];
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ V s_J[SPIN ? kMaxBondSlots : 1];
    __shared__ V s_cf[SPIN ? kSpinCoef : 1];
    __shared__ V s_inv_s[B], s_c_prev[B];
    __shared__ int s_skip;
    __shared__ uint32_t s_next;
    uint32_t loaded = 0xffffffffu;
    EpiDev ep{};
    // tiles after the first come from a counter in the wave's first unit (its words
    // 1 and 2: tiles handed out, CTAs done; zeroed by ms_reset_kernel and again by
    // the last CTA of each launch)
    unsigned int *wctr = reinterpret_cast<unsigned int *>(ws + units[0].off_st + (size_t)kMaxBlock * sizeof(ChainState)) + 1;
    for (uint32_t g = blockIdx.x; g < n_tiles;) {
        const uint32_t ui = tile_unit[g];
        const UnitView uv{units + ui, ws};
        const MsUnit &U = *uv.u;
        const int ju = j - U.j0;  // the unit's Lanczos step
        if (ui != loaded) {  // CTA-uniform: stage the unit's bonds, tlo and chain scalars
            __syncthreads();  // every thread is past its last read of the previous unit's data
            loaded = ui;
            if (SPIN) {
                for (uint32_t i = threadIdx.x; i < U.spin.nb; i += blockDim.x) {
                    s_bond[i] = U.spin.slots[i];
                    s_J[i] = spin_J<V>(U.spin)[i];
                }
                spin_stage_coef<V>(U.spin, s_cf);
            } else {
                const uint4 *src = sizeof(V) == 4 ? U.bl.slots_f32 : U.bl.slots_f64;
                for (int i = threadIdx.x; i < U.bl.nb; i += blockDim.x) s_bond[i] = src[i];
            }
            if (!CLT)
                for (uint32_t i = threadIdx.x; i <= U.s.lomask; i += blockDim.x) s_tlo[i] = __ldg(U.s.tlo + i);
            if (threadIdx.x == 0) {
                const ChainState *st = uv.st();
                int all = 1;
                for (int r = 0; r < B; ++r) all &= st[r].stopped;
                s_skip = all || ju < 1 || ju > U.m_max;
            }
            if (threadIdx.x < B) {
                const ChainState &c = uv.st()[threadIdx.x];
                s_inv_s[threadIdx.x] = (V)(1.0 / c.s_cur);
                s_c_prev[threadIdx.x] = ju > 1 ? (V)(c.beta_prev / c.s_prev) : (V)0;
            }
            ep.has_prev = ju > 1;
            __syncthreads();
        }
        if (!s_skip) {  // CTA-uniform
        const uint32_t k = g - U.tile0, D = U.s.D;
        const V *x = uv.vec<V>((ju - 1) & 1);
        V *y = uv.vec<V>(ju & 1);
        const V jsum4 = (V)U.bl.jsum4;
        DotAcc<V> apart[B];
        const uint32_t row0 = k * U.tile_rows;
        for (uint32_t p = 0; p < U.tile_rows; p += kRowThreads) {
            const uint32_t tt = row0 + p + threadIdx.x;
            if (row0 + p >= D) break;  // CTA-uniform
            const bool ok = tt < D;
            const uint32_t t[1] = {ok ? tt : D - 1};  // rows past the end recompute the last row, unstored
            if constexpr (SPIN) {
                V acc[B], diag;
                spin_row<V, B, C, false>(U.s, U.spin, s_tlo, nullptr, s_bond, s_J, s_cf, x, t[0], acc, diag);
                if (ok) epi_row<V, B, true>(ep, s_inv_s, s_c_prev, x, y, t[0], diag, acc, apart);
            } else {
                V acc[1][B], dsum[1] = {(V)0};
#pragma unroll
                for (int r = 0; r < B; ++r) acc[0][r] = (V)0;
                if (CLT) rows_clt<V, 1, B, C>(U.s, U.bl, s_bond, x, t, acc, dsum);
                else rows_cr<V, uint32_t, 1, B, C>(U.s, U.bl, s_bond, s_tlo, x, t, acc, dsum);
                if (ok) epi_row<V, B, true>(ep, s_inv_s, s_c_prev, x, y, t[0], jsum4 - dsum[0], acc[0], apart);
            }
        }
        if (tile_publish<V, B>(apart, uv.partials(), k, uv.counter(), U.n_tiles) && threadIdx.x < 32) {
            ChainState *st = uv.st();
            for (int r = 0; r < B; ++r) {
                const double v = tile_total<B>(uv.partials(), U.n_tiles, r);
                if (threadIdx.x == 0 && !st[r].stopped) {
                    st[r].alpha = v;
                    alpha[(size_t)(U.chain_base + r) * M + (ju - 1)] = v;
                }
            }
            if (threadIdx.x == 0) *uv.counter() = 0;
        }
        __syncthreads();
        }
        if (threadIdx.x == 0) s_next = atomicAdd(wctr, 1u) + gridDim.x;
        __syncthreads();
        g = s_next;
        __syncthreads();  // every thread has read s_next before thread 0 writes it again
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(wctr + 1, 1u) == gridDim.x - 1) {
            wctr[0] = 0;
            wctr[1] = 0;
        }
    }
}

// Step j: w = y - alpha_j q_j in place, beta_j = ||w||, breakdown test (as
// update_kernel of lanczos.cu, per unit).
template <typename V, int B>
__global__ void __launch_bounds__(kRowThreads)
ms_update_kernel(const MsUnit *__restrict__ units, const uint32_t *__restrict__ tile_unit, uint32_t n_tiles, int j,
                 int M, double *beta, char *ws)
{
    constexpr int W = 16 / (int)sizeof(V);
    constexpr int U_ = B > W ? B : W;  // values per thread and pass
    __shared__ V s_a[B];
    __shared__ int s_zero[B];
    __shared__ int s_skip;
    uint32_t loaded = 0xffffffffu;
    for (uint32_t g = blockIdx.x; g < n_tiles; g += gridDim.x) {
        const uint32_t ui = tile_unit[g];
        const UnitView uv{units + ui, ws};
        const MsUnit &U = *uv.u;
        const int ju = j - U.j0;  // the unit's Lanczos step
        if (ui != loaded) {
            __syncthreads();
            loaded = ui;
            if (threadIdx.x == 0) {
                const ChainState *st = uv.st();
                int all = 1;
                for (int r = 0; r < B; ++r) all &= st[r].stopped;
                s_skip = all || ju < 1 || ju > U.m_max;
            }
            if (threadIdx.x < B) {
                const ChainState &c = uv.st()[threadIdx.x];
                s_zero[threadIdx.x] = c.stopped;
                s_a[threadIdx.x] = c.stopped ? (V)0 : (V)(c.alpha / c.s_cur);
            }
            __syncthreads();
        }
        if (s_skip) continue;
        const uint32_t k = g - U.stile0, D = U.s.D;
        V *y = uv.vec<V>(ju & 1);
        const V *u = uv.vec<V>((ju - 1) & 1);
        V a[B];
        bool zero[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            a[r] = s_a[r];
            zero[r] = s_zero[r] != 0;
        }
        DotAcc<V> acc[B];
        const uint64_t e0 = (uint64_t)k * U.stream_rows * B;
        const uint64_t e1 = (uint64_t)min(D, (k + 1) * U.stream_rows) * B;
        const uint64_t full = e0 + (e1 - e0) / U_ * U_;
        for (uint64_t e = e0 + (uint64_t)threadIdx.x * U_; e < full; e += (uint64_t)kRowThreads * U_) {
            V yv[U_], xv[U_], w[U_];
            ld_vec<U_>(y + e, yv, true);
            ld_vec<U_>(u + e, xv, true);
#pragma unroll
            for (int q = 0; q < U_; ++q) {
                const int r = q % B;
                w[q] = zero[r] ? (V)0 : fma(-a[r], xv[q], yv[q]);
                acc[r].add(w[q], w[q]);
            }
            st_vec<U_>(y + e, w);
        }
        for (uint64_t e = full + threadIdx.x; e < e1; e += kRowThreads) {  // only with B = 1
            const V w = zero[0] ? (V)0 : fma(-a[0], u[e], y[e]);
            y[e] = w;
            acc[0].add(w, w);
        }
        if (tile_publish<V, B>(acc, uv.partials(), k, uv.counter(), U.n_stiles) && threadIdx.x < 32) {
            ChainState *st = uv.st();
            for (int r = 0; r < B; ++r) {
                const double bt = sqrt(tile_total<B>(uv.partials(), U.n_stiles, r));
                if (threadIdx.x == 0 && !st[r].stopped) {
                    ChainState &c = st[r];
                    if (ju < U.m_max) {
                        if (bt <= U.tau) {
                            c.stopped = 1;
                            c.m_eff = ju;
                        } else {
                            beta[(size_t)(U.chain_base + r) * M + (ju - 1)] = bt;
                            c.s_prev = c.s_cur;
                            c.s_cur = bt;
                            c.beta_prev = bt;
                        }
                    } else {
                        c.m_eff = U.m_max;
                    }
                }
            }
            if (threadIdx.x == 0) *uv.counter() = 0;
        }
        __syncthreads();
    }
}

// Chain states and reduction counters of every unit of the wave to zero (the
// counters must start at zero: the last tile of a unit is found by its ticket).
// Units with j0 == jstart only (a batch: every unit, jstart = 0).
__global__ void ms_reset_kernel(const MsUnit *__restrict__ units, uint32_t n_units, char *ws, int jstart)
{
    constexpr uint32_t words = (kMaxBlock * sizeof(ChainState) + 64) / sizeof(uint32_t);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_units * words; i += gridDim.x * blockDim.x) {
        const MsUnit &U = units[i / words];
        if (U.j0 != jstart) continue;
        uint32_t *p = reinterpret_cast<uint32_t *>(ws + U.off_st);
        p[i % words] = 0u;
    }
}

__global__ void ms_meff_kernel(const MsUnit *__restrict__ units, uint32_t n_units, int B, int *meff, char *ws)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_units * (uint32_t)B; i += gridDim.x * blockDim.x) {
        const MsUnit &U = units[i / B];
        const int r = (int)(i % B);
        if (r < U.nact) meff[U.chain_base + r] = reinterpret_cast<const ChainState *>(ws + U.off_st)[r].m_eff;
    }
}

template <int B> __host__ __device__ constexpr int ms_chunk() { return B >= 8 ? 4 : kBondChunk; }

template <typename V, int B> void *ms_hv_ptr(int kind)
{
    if (kind == kMsSpin) return (void *)ms_hv_kernel<V, kMsSpin, B, spin_chunk<B>()>;
    if (kind == kMsClt) return (void *)ms_hv_kernel<V, kMsClt, B, ms_chunk<B>()>;
    return (void *)ms_hv_kernel<V, kMsCr, B, ms_chunk<B>()>;
}

template <typename V, int B>
ftlm_status ms_run_typed(const MsWave &w, const MsUnit *units, const uint32_t *tile_unit,
                         const uint32_t *stile_unit, int M, int dist, char *ws, double *alpha, double *beta,
                         int *meff, int num_sms, cudaStream_t stream)
{
    const size_t smem = w.kind == kMsClt ? 0 : ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
    void *hv = ms_hv_ptr<V, B>(w.kind);
    int oh = 1, occ_start = 1, occ_upd = 1;
    FTLM_CUDA(kernel_occupancy(hv, kRowThreads, smem, smem != 0, &oh));
    FTLM_CUDA(kernel_occupancy((const void *)ms_start_kernel<V, B>, kRowThreads, 0, false, &occ_start));
    FTLM_CUDA(kernel_occupancy((const void *)ms_update_kernel<V, B>, kRowThreads, 0, false, &occ_upd));
    auto grid = [&](int occ) { return (int)std::min<uint64_t>(w.n_tiles, (uint64_t)num_sms * occ); };
    auto sgrid = [&](int occ) { return (int)std::min<uint64_t>(w.n_stiles, (uint64_t)num_sms * occ); };
    {
        const uint32_t words = (kMaxBlock * sizeof(ChainState) + 64) / sizeof(uint32_t);
        const int g = (int)std::min<uint64_t>(((uint64_t)w.n_units * words + 255) / 256, (uint64_t)num_sms * 4);
        ms_reset_kernel<<<g, 256, 0, stream>>>(units, w.n_units, ws, 0);
        note_launch();
    }
    ms_start_kernel<V, B><<<sgrid(occ_start), kRowThreads, 0, stream>>>(units, stile_unit, w.n_stiles, dist, ws, 0);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    for (int j = 1; j <= w.m_max; ++j) {
        void *tok = profile_begin(kProfHv, stream, B);
        uint32_t nt = w.n_tiles;
        int jj = j, MM = M;
        void *args[] = {(void *)&units, (void *)&tile_unit, (void *)&nt, (void *)&jj, (void *)&MM, (void *)&alpha,
                        (void *)&ws};
        FTLM_CUDA(cudaLaunchKernel(hv, dim3(grid(oh)), dim3(kRowThreads), args, smem, stream));
        note_launch();
        profile_end(tok, stream);
        tok = profile_begin(kProfUpdate, stream);
        ms_update_kernel<V, B><<<sgrid(occ_upd), kRowThreads, 0, stream>>>(units, stile_unit, w.n_stiles, j, M,
                                                                            beta, ws);
        note_launch();
        profile_end(tok, stream);
        FTLM_CUDA(cudaGetLastError());
    }
    ms_meff_kernel<<<(w.n_units * B + 255) / 256, 256, 0, stream>>>(units, w.n_units, B, meff, ws);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V>
ftlm_status ms_run_v(const MsWave &w, int B, const MsUnit *units, const uint32_t *tu, const uint32_t *su, int M,
                     int dist, char *ws, double *alpha, double *beta, int *meff, int num_sms, cudaStream_t stream)
{
    switch (B) {
    case 16: return ms_run_typed<V, 16>(w, units, tu, su, M, dist, ws, alpha, beta, meff, num_sms, stream);
    case 8: return ms_run_typed<V, 8>(w, units, tu, su, M, dist, ws, alpha, beta, meff, num_sms, stream);
    case 4: return ms_run_typed<V, 4>(w, units, tu, su, M, dist, ws, alpha, beta, meff, num_sms, stream);
    default: return ms_run_typed<V, 1>(w, units, tu, su, M, dist, ws, alpha, beta, meff, num_sms, stream);
    }
}

// ---- single launches for a continuous flow (flow.cu) -------------------------
template <typename V, int B>
ftlm_status flow_start_typed(const MsUnit *units, uint32_t n_units, const uint32_t *stile_unit, uint32_t n_stiles,
                             int jstart, int dist, char *ws, int num_sms, cudaStream_t stream)
{
    int occ = 1;
    FTLM_CUDA(kernel_occupancy((const void *)ms_start_kernel<V, B>, kRowThreads, 0, false, &occ));
    const uint32_t words = (kMaxBlock * sizeof(ChainState) + 64) / sizeof(uint32_t);
    const int g = (int)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)n_units * words + 255) / 256,
                                                                (uint64_t)num_sms * 4));
    ms_reset_kernel<<<g, 256, 0, stream>>>(units, n_units, ws, jstart);
    note_launch();
    const int gs = (int)std::max<uint64_t>(1, std::min<uint64_t>(n_stiles, (uint64_t)num_sms * occ));
    ms_start_kernel<V, B><<<gs, kRowThreads, 0, stream>>>(units, stile_unit, n_stiles, dist, ws, jstart);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V, int B>
ftlm_status flow_hv_typed(int kind, const MsUnit *units, const uint32_t *tile_unit, uint32_t n_tiles, int j, int M,
                          double *alpha, char *ws, int num_sms, cudaStream_t stream)
{
    const size_t smem = kind == kMsClt ? 0 : ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
    void *hv = ms_hv_ptr<V, B>(kind);
    int oh = 1;
    FTLM_CUDA(kernel_occupancy(hv, kRowThreads, smem, smem != 0, &oh));
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, (uint64_t)num_sms * oh));
    void *args[] = {(void *)&units, (void *)&tile_unit, (void *)&n_tiles, (void *)&j, (void *)&M, (void *)&alpha,
                    (void *)&ws};
    void *tok = profile_begin(kProfHv, stream, B);
    FTLM_CUDA(cudaLaunchKernel(hv, dim3(grid), dim3(kRowThreads), args, smem, stream));
    note_launch();
    profile_end(tok, stream);
    return FTLM_OK;
}

template <typename V, int B>
ftlm_status flow_update_typed(const MsUnit *units, const uint32_t *stile_unit, uint32_t n_stiles, int j, int M,
                              double *beta, char *ws, int num_sms, cudaStream_t stream)
{
    int occ = 1;
    FTLM_CUDA(kernel_occupancy((const void *)ms_update_kernel<V, B>, kRowThreads, 0, false, &occ));
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(n_stiles, (uint64_t)num_sms * occ));
    void *tok = profile_begin(kProfUpdate, stream);
    ms_update_kernel<V, B><<<grid, kRowThreads, 0, stream>>>(units, stile_unit, n_stiles, j, M, beta, ws);
    note_launch();
    profile_end(tok, stream);
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

#define FTLM_FLOW_DISPATCH(FN, ...)                                                         \
    switch (B) {                                                                           \
    case 16: return dtype == FTLM_F32 ? FN<float, 16>(__VA_ARGS__) : FN<double, 16>(__VA_ARGS__); \
    case 8: return dtype == FTLM_F32 ? FN<float, 8>(__VA_ARGS__) : FN<double, 8>(__VA_ARGS__);    \
    case 4: return dtype == FTLM_F32 ? FN<float, 4>(__VA_ARGS__) : FN<double, 4>(__VA_ARGS__);    \
    default: return dtype == FTLM_F32 ? FN<float, 1>(__VA_ARGS__) : FN<double, 1>(__VA_ARGS__);   \
    }

}  // namespace

ftlm_status ms_flow_start(ftlm_dtype dtype, int B, const MsUnit *units, uint32_t n_units, const uint32_t *stile_unit,
                          uint32_t n_stiles, int jstart, int dist, char *ws, int num_sms, cudaStream_t stream)
{
    FTLM_FLOW_DISPATCH(flow_start_typed, units, n_units, stile_unit, n_stiles, jstart, dist, ws, num_sms, stream)
}

ftlm_status ms_flow_hv(ftlm_dtype dtype, int B, int kind, const MsUnit *units, const uint32_t *tile_unit,
                       uint32_t n_tiles, int j, int M, double *alpha, char *ws, int num_sms, cudaStream_t stream)
{
    FTLM_FLOW_DISPATCH(flow_hv_typed, kind, units, tile_unit, n_tiles, j, M, alpha, ws, num_sms, stream)
}

ftlm_status ms_flow_update(ftlm_dtype dtype, int B, const MsUnit *units, const uint32_t *stile_unit, uint32_t n_stiles,
                           int j, int M, double *beta, char *ws, int num_sms, cudaStream_t stream)
{
    FTLM_FLOW_DISPATCH(flow_update_typed, units, stile_unit, n_stiles, j, M, beta, ws, num_sms, stream)
}

ftlm_status ms_run_wave(const MsWave &w, ftlm_dtype dtype, int B, const MsUnit *units, const uint32_t *tile_unit,
                        const uint32_t *stile_unit, int M, int dist, char *ws, double *alpha, double *beta,
                        int *meff, int num_sms, cudaStream_t stream)
{
    if (!w.n_tiles) return FTLM_OK;
    return dtype == FTLM_F32
               ? ms_run_v<float>(w, B, units, tile_unit, stile_unit, M, dist, ws, alpha, beta, meff, num_sms, stream)
               : ms_run_v<double>(w, B, units, tile_unit, stile_unit, M, dist, ws, alpha, beta, meff, num_sms,
                                  stream);
}

}  // namespace ftlm
