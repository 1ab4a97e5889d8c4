// H.v gather (step a3), Eq. 12 with the ladder coefficients of Eq. 13-14 at
// s = 1/2, and the Lanczos epilogue fused into the same launch (step a4).
//
// One thread owns one output row t (the row-wise gather of Sec. 2): it recovers
// its label n_t, and for every bond whose two spins are antiparallel in n_t it
// exchanges them, ranks the resulting source label k and gathers (J_b/2) x[k].
// The diagonal sum_b J_b m_i m_j equals sum_b J_b/4 - sum_{b antiparallel} J_b/2,
// so it is accumulated alongside the gathers.  Each thread writes one y[t]; there
// are no atomics.
//
// Bonds are warp-uniform (a kernel parameter read through the constant bank), and
// the 32 rows of a warp are 32 consecutive sector indices, i.e. 32 consecutive
// labels in increasing order that differ only in their lowest bits.  For a bond
// on high sites the exchange therefore shifts all 32 ranks by the same amount and
// the warp's gather is one contiguous 128-byte line; bonds on low sites land within
// a few lines of the warp's own rows.  The grid is persistent (a multiple of the
// SM count) and walks the rows in order, so at any moment every bond's gather
// stream sits in a narrow window of x and the windows stay L2-resident.
//
// Two rank strategies:
//   CLT  label n_t = basis[t]; rank(n') = C_b + popc(M_b & (2^j - 1)) with
//        b = n' >> 5, j = n' & 31 (Eq. 19-20, Algorithm 2); {M_b, C_b} is one
//        8-byte entry.
//   CR   rank(n) = thi[n >> L] + tlo[n & (2^L-1)] (Algorithm 1 with the L low
//        digits and the N-L high digits each collapsed into one table lookup);
//        the row label is recovered by the inverse map (binary search of thi,
//        then ulo).  tlo (2^L x 16 bit) is staged in shared memory; thi is read
//        through L1 and is warp-uniform for almost every row.  A bond with both
//        sites in one block changes only that block's lookup: the other half of
//        the rank is the row's own.
//
// Block H.v (B vectors, interleaved: element (t, r) at t * B + r).  The row's rank
// work is done once and every antiparallel bond gathers B contiguous values
// (32 bytes, one DRAM sector, for B = 8 in FP32), so the index arithmetic and the
// table lookups are shared by the B vectors -- the batched scheme of Sec. 3.4.
//
// Lanczos epilogue (Paige's ordering), per chain r of the block.  Per-thread
// partial dot products use DotAcc (exact products, two-float compensated sums for
// FP32 vectors); block and grid sums are FP64.  The stored vector
// u_j is un-normalized, q_j = u_j / s_j.  With x = u_j and the in-place buffer
// holding u_{j-1}:
//   y[t] = (H u_j)[t] / s_j - (beta_{j-1} / s_{j-1}) u_{j-1}[t]     (overwrites u_{j-1})
//   alpha partial += q_j[t] y[t]                                    (FP64)
// The last block adds the per-block partials in a fixed order and stores alpha_j.
#include <algorithm>
#include <cstdlib>

#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "vec.cuh"

namespace ftlm {

namespace {

struct EpiDev {
    ChainState *st;
    double *partials;
    unsigned int *counter;
    double *alpha_out;
    int alpha_stride;
    int has_prev;
};

// J/2 of a bond slot in the vector type.
template <typename V> __device__ __forceinline__ V slot_jh(const uint4 &e);
template <> __device__ __forceinline__ float slot_jh<float>(const uint4 &e) { return __uint_as_float(e.z); }
template <> __device__ __forceinline__ double slot_jh<double>(const uint4 &e)
{
    return __hiloint2double((int)e.w, (int)e.z);
}

// Bonds per chunk: 8, or 4 when each gather brings 8 or more values.
template <int B> __host__ __device__ constexpr int chunk_of() { return B >= 8 ? 4 : kBondChunk; }

// Bond data of one chunk, read once and applied to every row of the thread.
template <typename V, int C>
struct Chunk {
    uint32_t mlo[C], mhi[C];
    V jh[C];
};

template <typename V, int C>
__device__ __forceinline__ void load_chunk(const uint4 *s_bond, int b0, Chunk<V, C> &c)
{
#pragma unroll
    for (int q = 0; q < C; ++q) {
        const uint4 e = s_bond[b0 + q];  // same address in every lane: a broadcast
        c.mlo[q] = e.x;
        c.mhi[q] = e.y;
        c.jh[q] = slot_jh<V>(e);
    }
}

// Gather the chunk's antiparallel terms of RT rows (predicated loads, all issued
// before the first use) and accumulate them into acc[row][vector].
template <typename V, int RT, int B, int C>
__device__ __forceinline__ void gather_accumulate(const V *__restrict__ x, const Chunk<V, C> &c,
                                                  const bool (&aa)[RT][C], const uint32_t (&kk)[RT][C],
                                                  V (&acc)[RT][B], V (&dsum)[RT])
{
    V xv[RT][C][B];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < C; ++q) {
            if (aa[i][q]) {
                ld_vec<B>(x + (size_t)kk[i][q] * B, xv[i][q], false);
            } else {
#pragma unroll
                for (int r = 0; r < B; ++r) xv[i][q][r] = (V)0;
            }
        }
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < C; ++q)
            if (aa[i][q]) {
#pragma unroll
                for (int r = 0; r < B; ++r) acc[i][r] = fma(c.jh[q], xv[i][q][r], acc[i][r]);
                dsum[i] += c.jh[q];
            }
}

// Inverse map t -> (h, l) through the digit-block tables: the coarse index bounds
// h to [hs[t >> kHsShift], hs[(t >> kHsShift) + 1]]; a binary search of thi finds
// the last h with thi[h] <= t; the low pattern is entry t - thi[h] of popcount
// group K - popcount(h).
__device__ __forceinline__ void unrank_hl(const SectorTables &s, uint32_t t, uint32_t &h, uint32_t &l,
                                          uint32_t &r_hi, uint32_t &r_lo)
{
    const uint32_t kc = t >> kHsShift;
    uint32_t lo = __ldg(s.hs + kc), hi = __ldg(s.hs + kc + 1) + 1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(s.thi + mid) <= t) lo = mid;
        else hi = mid;
    }
    h = lo;
    r_hi = __ldg(s.thi + h);
    r_lo = t - r_hi;
    l = __ldg(s.ulo + __ldg(s.uoff + (s.K - __popc(h))) + r_lo);
}

// Row sums of RT output rows (CR): sum over antiparallel bonds of (J_b/2) x[k_b]
// in acc, sum of their J_b/2 in dsum.
template <typename V, typename Lbl, int RT, int B>
__device__ __forceinline__ void rows_cr(const SectorTables &s, const BondList &bl, const uint4 *s_bond,
                                        const uint16_t *s_tlo, const V *__restrict__ x,
                                        const uint32_t (&t)[RT], V (&acc)[RT][B], V (&dsum)[RT])
{
    constexpr int C = chunk_of<B>();
    uint32_t h[RT], l[RT], r_hi[RT], r_lo[RT];
#pragma unroll
    for (int i = 0; i < RT; ++i) unrank_hl(s, t[i], h[i], l[i], r_hi[i], r_lo[i]);
    Chunk<V, C> c;
    bool aa[RT][C];
    uint32_t kk[RT][C];
    const int e_lo = bl.n_lo, e_hi = bl.n_lo + bl.n_hi;
    for (int b0 = 0; b0 < e_lo; b0 += C) {  // both sites in the low block
        load_chunk(s_bond, b0, c);
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const uint32_t m = c.mlo[q], xm = l[i] & m;
                aa[i][q] = (xm != 0u) & (xm != m);
                kk[i][q] = r_hi[i] + s_tlo[l[i] ^ m];
            }
        gather_accumulate<V, RT, B, C>(x, c, aa, kk, acc, dsum);
    }
    for (int b0 = e_lo; b0 < e_hi; b0 += C) {  // both sites in the high block
        load_chunk(s_bond, b0, c);
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const uint32_t m = c.mhi[q], xm = h[i] & m;
                aa[i][q] = (xm != 0u) & (xm != m);
                kk[i][q] = __ldg(s.thi + (h[i] ^ m)) + r_lo[i];
            }
        gather_accumulate<V, RT, B, C>(x, c, aa, kk, acc, dsum);
    }
    for (int b0 = e_hi; b0 < bl.nb; b0 += C) {  // any bond
        load_chunk(s_bond, b0, c);
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const Lbl n = ((Lbl)h[i] << s.L) | l[i];
#pragma unroll
            for (int q = 0; q < C; ++q) {
                Lbl m = c.mlo[q];
                if constexpr (sizeof(Lbl) == 8) m |= (Lbl)c.mhi[q] << 32;
                const Lbl xm = n & m, nn = n ^ m;
                aa[i][q] = (xm != 0) & (xm != m);
                kk[i][q] = __ldg(s.thi + (uint32_t)(nn >> s.L)) + s_tlo[(uint32_t)nn & s.lomask];
            }
        }
        gather_accumulate<V, RT, B, C>(x, c, aa, kk, acc, dsum);
    }
}

// Row sums of RT output rows (CLT, Algorithm 2 per exchanged label).
template <typename V, int RT, int B>
__device__ __forceinline__ void rows_clt(const SectorTables &s, const BondList &bl, const uint4 *s_bond,
                                         const V *__restrict__ x, const uint32_t (&t)[RT], V (&acc)[RT][B],
                                         V (&dsum)[RT])
{
    constexpr int C = chunk_of<B>();
    uint32_t n[RT];
#pragma unroll
    for (int i = 0; i < RT; ++i) n[i] = __ldcs(s.basis + t[i]);
    Chunk<V, C> c;
    bool aa[RT][C];
    uint32_t kk[RT][C];
    for (int b0 = 0; b0 < bl.nb; b0 += C) {
        load_chunk(s_bond, b0, c);
        uint2 e2[RT][C];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const uint32_t m = c.mlo[q], xm = n[i] & m;
                aa[i][q] = (xm != 0u) & (xm != m);
                e2[i][q] = aa[i][q] ? __ldg(s.clt + ((n[i] ^ m) >> 5)) : make_uint2(0u, 0u);
            }
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const uint32_t nn = n[i] ^ c.mlo[q];
                kk[i][q] = e2[i][q].y + __popc(e2[i][q].x & ((1u << (nn & 31u)) - 1u));
            }
        gather_accumulate<V, RT, B, C>(x, c, aa, kk, acc, dsum);
    }
}

// One warp owns a tile of 32 RT consecutive rows; lane l handles rows
// tile_base + l + 32 i (i < RT).  Tiles are dealt to warps round-robin, so the
// whole grid works on one contiguous window of rows at a time.
// Resident CTAs per SM the compiler must allow for (register budget).  Single
// vectors with up to 2 rows per thread keep a small register footprint (6 CTAs of
// 256 threads, the shared-memory limit of the CR kernel); 4 rows per thread and
// blocks of 4-8 vectors get at least 3 CTAs per SM (fewer starve the loads);
// 16-wide blocks keep all their registers (a cap spills).
template <int RT, int B> __host__ __device__ constexpr int min_ctas()
{
    return B >= 16 ? 1 : (B >= 4 || RT >= 4 ? 3 : 6);
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS, int RT, int B>
__global__ void __launch_bounds__(kRowThreads, min_ctas<RT, B>())
hv_kernel(const SectorTables s, const BondList bl, const V *__restrict__ x, V *y, const EpiDev ep)
{
    extern __shared__ uint16_t s_tlo[];
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ V s_inv_s[B], s_c_prev[B];  // per-chain scalars of the epilogue
    if (LANCZOS) {
        bool all_stopped = true;
#pragma unroll
        for (int r = 0; r < B; ++r) all_stopped &= ep.st[r].stopped != 0;
        if (all_stopped) return;  // every chain of the block ended: grid-uniform
        if (threadIdx.x < B) {
            const ChainState &st = ep.st[threadIdx.x];
            s_inv_s[threadIdx.x] = (V)(1.0 / st.s_cur);
            s_c_prev[threadIdx.x] = ep.has_prev ? (V)(st.beta_prev / st.s_prev) : (V)0;
        }
    }
    {
        const uint4 *src = sizeof(V) == 4 ? bl.slots_f32 : bl.slots_f64;
        for (int i = threadIdx.x; i < bl.nb; i += blockDim.x) s_bond[i] = src[i];
    }
    if (!CLT)
        for (uint32_t i = threadIdx.x; i <= s.lomask; i += blockDim.x) s_tlo[i] = __ldg(s.tlo + i);
    __syncthreads();
    const V jsum4 = (V)bl.jsum4;
    DotAcc<V> apart[B];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t tile_rows = 32u * RT;
    const uint32_t ntiles = (uint32_t)(((uint64_t)s.D + tile_rows - 1) / tile_rows);
    for (uint32_t tile = warp; tile < ntiles; tile += nwarps) {
        uint32_t t[RT];
        bool ok[RT];
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const uint32_t tt = tile * tile_rows + 32u * i + lane;
            ok[i] = tt < s.D;
            t[i] = ok[i] ? tt : s.D - 1;  // rows past the end recompute the last row, unstored
        }
        V acc[RT][B], dsum[RT];
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            dsum[i] = (V)0;
#pragma unroll
            for (int r = 0; r < B; ++r) acc[i][r] = (V)0;
        }
        if (CLT) rows_clt<V, RT, B>(s, bl, s_bond, x, t, acc, dsum);
        else rows_cr<V, Lbl, RT, B>(s, bl, s_bond, s_tlo, x, t, acc, dsum);
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            if (!ok[i]) continue;
            V xt[B], out[B];
            ld_vec<B>(x + (size_t)t[i] * B, xt, false);
            const V diag = jsum4 - dsum[i];
            if (LANCZOS) {
                V up[B];
                if (ep.has_prev) ld_vec<B>(y + (size_t)t[i] * B, up, true);
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const V inv_s = s_inv_s[r];
                    const V hv = fma(diag, xt[r], acc[i][r]);
                    out[r] = ep.has_prev ? fma(-s_c_prev[r], up[r], hv * inv_s) : hv * inv_s;
                    apart[r].add(xt[r] * inv_s, out[r]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < B; ++r) out[r] = fma(diag, xt[r], acc[i][r]);
            }
            st_vec<B>(y + (size_t)t[i] * B, out);
        }
    }
    if (LANCZOS) {
        __shared__ double s_part[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            const double part = block_sum<kRowThreads>(apart[r].value());
            if (threadIdx.x == 0) s_part[r] = part;
        }
        __syncthreads();
        bool last = false;
        {
            __shared__ bool s_last;
            if (threadIdx.x == 0) {
#pragma unroll
                for (int r = 0; r < B; ++r) ep.partials[(size_t)blockIdx.x * B + r] = s_part[r];
                __threadfence();
                s_last = atomicAdd(ep.counter, 1u) == gridDim.x - 1;
            }
            __syncthreads();
            last = s_last;
        }
        if (last && threadIdx.x < 32) {
            for (int r = 0; r < B; ++r) {
                double v = 0.0;
                for (int g = threadIdx.x; g < (int)gridDim.x; g += 32) v += __ldcg(ep.partials + (size_t)g * B + r);
                v = warp_sum(v);
                if (threadIdx.x == 0 && !ep.st[r].stopped) {
                    ep.st[r].alpha = v;
                    ep.alpha_out[(size_t)r * ep.alpha_stride] = v;
                }
            }
            if (threadIdx.x == 0) *ep.counter = 0;
        }
    }
}

// Rows per thread (RT) for single vectors.  Measured on GB300 (icosidodecahedron,
// FP32): CR is fastest with 2 rows per thread (its rank tables are L1/shared-memory
// resident and the bond chunk is reused across rows), CLT with 1 (its two dependent
// gathers per bond already fill the load queues).  Blocks of vectors use 1.
// FTLM_HV_ROWS = 1, 2 or 4 overrides the single-vector choice.
int rows_per_thread(bool clt)
{
    static const int over = [] {
        const char *e = getenv("FTLM_HV_ROWS");
        const int v = e ? atoi(e) : 0;
        return (v == 1 || v == 2 || v == 4) ? v : 0;
    }();
    return over ? over : (clt ? 1 : 2);
}

// Cap on resident CTAs per SM used for the H.v grid (FTLM_HV_CTAS, default: no cap).
// Fewer CTAs shrink the window of rows in flight and with it the L2 working set of
// the gather streams.
int hv_cta_cap()
{
    static const int cap = [] {
        const char *e = getenv("FTLM_HV_CTAS");
        const int v = e ? atoi(e) : 0;
        return v > 0 ? v : kMaxBlocksPerSm;
    }();
    return cap;
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS, int RT, int B>
ftlm_status launch(const ftlm_basis *b, const V *x, V *y, const EpiDev &ep, cudaStream_t stream)
{
    static int occ = -1;  // resident blocks per SM for this instantiation
    const size_t smem = CLT ? 0 : ((size_t)1 << b->L) * sizeof(uint16_t);
    auto kern = hv_kernel<V, Lbl, CLT, LANCZOS, RT, B>;
    if (occ < 0) {
        const size_t smem_max = CLT ? 0 : ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
        FTLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRowThreads, smem_max));
    }
    const int grid = row_grid(b, (b->D + RT - 1) / RT, std::min(occ, hv_cta_cap()));
    void *tok = profile_begin(kProfHv, stream, B);
    kern<<<grid, kRowThreads, smem, stream>>>(b->tables(), CLT ? b->bonds_clt : b->bonds_cr, x, y, ep);
    profile_end(tok, stream);
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS>
ftlm_status launch_b(const ftlm_basis *b, int B, const void *x, void *y, const EpiDev &ep, cudaStream_t stream)
{
    const V *xv = (const V *)x;
    V *yv = (V *)y;
    switch (B) {
    case 4: return launch<V, Lbl, CLT, LANCZOS, 1, 4>(b, xv, yv, ep, stream);
    case 8: return launch<V, Lbl, CLT, LANCZOS, 1, 8>(b, xv, yv, ep, stream);
    case 16: return launch<V, Lbl, CLT, LANCZOS, 1, 16>(b, xv, yv, ep, stream);
    default: break;
    }
    switch (rows_per_thread(CLT)) {
    case 1: return launch<V, Lbl, CLT, LANCZOS, 1, 1>(b, xv, yv, ep, stream);
    case 4: return launch<V, Lbl, CLT, LANCZOS, 4, 1>(b, xv, yv, ep, stream);
    default: return launch<V, Lbl, CLT, LANCZOS, 2, 1>(b, xv, yv, ep, stream);
    }
}

template <typename V, bool LANCZOS>
ftlm_status launch_mode(const ftlm_basis *b, int B, const void *x, void *y, const EpiDev &ep,
                        cudaStream_t stream)
{
    if (b->mode == FTLM_RANK_CLT) return launch_b<V, uint32_t, true, LANCZOS>(b, B, x, y, ep, stream);
    if (b->N <= 32) return launch_b<V, uint32_t, false, LANCZOS>(b, B, x, y, ep, stream);
    return launch_b<V, uint64_t, false, LANCZOS>(b, B, x, y, ep, stream);
}

template <typename V>
ftlm_status launch_typed(const ftlm_basis *b, int B, const void *x, void *y, const LanczosHv *epi,
                         cudaStream_t stream)
{
    EpiDev ep{};
    if (epi) {
        ep.st = epi->st;
        ep.partials = epi->partials;
        ep.counter = epi->counter;
        ep.alpha_out = epi->alpha_out;
        ep.alpha_stride = epi->alpha_stride;
        ep.has_prev = epi->j > 1;
        return launch_mode<V, true>(b, B, x, y, ep, stream);
    }
    return launch_mode<V, false>(b, B, x, y, ep, stream);
}

}  // namespace

bool valid_block(int B) { return B == 1 || B == 4 || B == 8 || B == 16; }

ftlm_status launch_hv(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y,
                      const LanczosHv *epi, cudaStream_t stream)
{
    return dtype == FTLM_F32 ? launch_typed<float>(b, B, x, y, epi, stream)
                             : launch_typed<double>(b, B, x, y, epi, stream);
}

}  // namespace ftlm

namespace {
ftlm_status check_hv_args(const ftlm_basis *b, ftlm_dtype dtype, const void *x_dev, void *y_dev)
{
    if (!b) return ftlm::fail(FTLM_EINVAL, "NULL basis");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return ftlm::fail(FTLM_EINVAL, "bad dtype");
    if (!x_dev || !y_dev) return ftlm::fail(FTLM_EINVAL, "NULL vector");
    if (x_dev == y_dev) return ftlm::fail(FTLM_EINVAL, "x and y must not overlap");
    if (((uintptr_t)x_dev | (uintptr_t)y_dev) & 15u) return ftlm::fail(FTLM_EINVAL, "vectors must be 16-byte aligned");
    return FTLM_OK;
}
}  // namespace

extern "C" ftlm_status ftlm_hv(const ftlm_basis *b, ftlm_dtype dtype, const void *x_dev, void *y_dev,
                               void *stream)
{
    ftlm_status s = check_hv_args(b, dtype, x_dev, y_dev);
    if (s != FTLM_OK) return s;
    return ftlm::launch_hv(b, dtype, 1, x_dev, y_dev, nullptr, (cudaStream_t)stream);
}

extern "C" ftlm_status ftlm_hv_block(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x_dev,
                                     void *y_dev, void *stream)
{
    ftlm_status s = check_hv_args(b, dtype, x_dev, y_dev);
    if (s != FTLM_OK) return s;
    if (!ftlm::valid_block(B)) return ftlm::fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    return ftlm::launch_hv(b, dtype, B, x_dev, y_dev, nullptr, (cudaStream_t)stream);
}
