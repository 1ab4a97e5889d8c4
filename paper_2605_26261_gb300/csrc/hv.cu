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
// Bonds are warp-uniform (staged once per CTA in shared memory and read as
// broadcasts), and the 32 rows of a warp are 32 consecutive sector indices, i.e.
// 32 consecutive labels in increasing order that differ only in their lowest bits.  For a bond
// on high sites the exchange therefore shifts all 32 ranks by the same amount and
// the warp's gather is one contiguous 128-byte line; bonds on low sites land within
// a few lines of the warp's own rows.  The grid is persistent (a multiple of the
// SM count) and walks the rows in order, so at any moment every bond's gather
// stream sits in a narrow window of x and the windows stay L2-resident.  CLT
// launches and plain H.v deal 32-row tiles to warps round-robin; CR Lanczos
// launches hand them out from a counter, which keeps the warps on one frontier
// of rows (they drift apart under the round-robin order, and the union of the
// gather windows outgrows L2: 20 % fewer DRAM bytes, 25 % less time on the N = 30
// icosahedral sector).  Their alpha sums are then finished per tile (epi.cuh).
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
// The Lanczos epilogue (Paige's ordering) runs in the same launch (epi.cuh).
#include <algorithm>
#include <cstdlib>

#include "epi.cuh"
#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "vec.cuh"
#include "rows.cuh"

namespace ftlm {

namespace {

// Resident CTAs per SM the compiler must allow for (register budget).  Single
// vectors with up to 2 rows per thread keep a small register footprint (6 CTAs of
// 256 threads, the shared-memory limit of the CR kernel); 4 rows per thread and
// blocks of 4-8 vectors get at least 3 CTAs per SM (fewer starve the loads), 2 with
// 8-bond chunks of 8-wide blocks (their 16 gathers per row in flight carry it);
// 16-wide blocks keep all their registers (a cap spills).  FP64 vectors need about
// twice the registers: 4 CTAs for single vectors (3 with 2 rows per thread, 2 with
// 4), 2 for blocks of 4 and 1 for wider blocks, none of them spilling.
// Build option FTLM_B8_MIN_CTAS: the FP32 cut for 8-wide blocks with chunks of 4.
#ifndef FTLM_B8_MIN_CTAS
#define FTLM_B8_MIN_CTAS 3
#endif

template <typename V, int RT, int B, int C> __host__ __device__ constexpr int min_ctas()
{
    if (sizeof(V) == 8)  // FP64 accumulators and gathers take twice the registers
        return B >= 8 ? 1 : (B >= 4 ? 2 : (RT >= 4 ? 2 : (RT >= 2 ? 3 : 4)));
    return B >= 16 ? 1
                   : (B >= 8 && C >= 8 ? 2
                                       : (B >= 8 && C <= 2 ? 4 : (B >= 8 ? FTLM_B8_MIN_CTAS : (B >= 4 || RT >= 4 ? 3 : 6))));
}

// EPI: kPlain (y = H x) or kLanczos (fused Lanczos epilogue with alpha).
enum { kPlain = 0, kLanczos = 1 };

template <typename V, typename Lbl, bool CLT, int EPI, int RT, int B, int C>
__global__ void __launch_bounds__(kRowThreads, min_ctas<V, RT, B, C>())
hv_kernel(const SectorTables s, const BondList bl, const V *__restrict__ x, V *y, const EpiDev ep)
{
    constexpr bool LANCZOS = EPI != kPlain;
    // CR Lanczos launches take their tiles in dynamic order (their gathers gain the
    // most from a narrow frontier of rows) and store per-tile alpha sums
    constexpr bool TILES = LANCZOS && !CLT;
    extern __shared__ uint16_t s_tlo[];
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ V s_inv_s[B], s_c_prev[B];  // per-chain scalars of the epilogue
    if (LANCZOS && epi_begin<V, B>(ep, s_inv_s, s_c_prev)) return;
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
    // the rows of one tile: rank work, gathers and the epilogue of the mode
    auto do_tile = [&](uint32_t tile) {
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
        if (CLT) rows_clt<V, RT, B, C>(s, bl, s_bond, x, t, acc, dsum);
        else rows_cr<V, Lbl, RT, B, C>(s, bl, s_bond, s_tlo, x, t, acc, dsum);
        if constexpr (TILES) {
            DotAcc<V> tacc[B];
#pragma unroll
            for (int i = 0; i < RT; ++i)
                if (ok[i]) epi_row<V, B, true>(ep, s_inv_s, s_c_prev, x, y, t[i], jsum4 - dsum[i], acc[i], tacc);
            store_tile<V, B>(ep, tile, tacc);
        } else {
#pragma unroll
            for (int i = 0; i < RT; ++i)
                if (ok[i]) epi_row<V, B, LANCZOS>(ep, s_inv_s, s_c_prev, x, y, t[i], jsum4 - dsum[i], acc[i], apart);
        }
    };
    for (uint32_t tile = warp; tile < ntiles;) {
        // claim the next tile now; its atomic completes while this tile's rows run
        const uint32_t claim = TILES ? claim_tile(ep) : 0u;
        do_tile(tile);
        tile = TILES ? claimed_tile(claim, nwarps) : tile + nwarps;
    }
    if (TILES) tiles_done(ep, nwarps);
    else if (LANCZOS) epi_end<V, B, kRowThreads>(ep, apart);
}

// alpha_j of a dynamically ordered launch from its per-tile sums: block b adds a
// fixed range of tiles (each thread its tiles in order), then the block trees and
// the last block's sum over the blocks in order (epi_end).  The grid depends only
// on the tile count, so alpha_j is reproducible.
template <int B>
__global__ void __launch_bounds__(kRowThreads) tile_alpha_kernel(const EpiDev ep, uint32_t ntiles)
{
    bool all_stopped = true;
#pragma unroll
    for (int r = 0; r < B; ++r) all_stopped &= ep.st[r].stopped != 0;
    if (all_stopped) return;  // as the H.v launch: uniform over the grid
    const uint32_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    const uint32_t t0 = min(ntiles, blockIdx.x * per), t1 = min(ntiles, t0 + per);
    DotAcc<double> a[B];
    for (uint32_t t = t0 + threadIdx.x; t < t1; t += blockDim.x)
#pragma unroll
        for (int r = 0; r < B; ++r) a[r].v += __ldcg(ep.tile_part + (size_t)t * B + r);
    epi_end<double, B, kRowThreads>(ep, a);
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

// Split Lanczos H.v (see HiWalk, LoWalk): used when the basis asks for it, or
// under FTLM_HV_AUTO for blocks of vectors of at least kSplitMinBytes32 (FP32;
// kSplitMinBytes32Rows for rows of 32 bytes or more) or kSplitMinBytes64 (FP64) of
// sectors with at least kSplitMinHiBonds high-high bonds.  Measured on GB300 (H.v
// step, one walk -> split), N = 30 icosidodecahedral sectors (26 of 60 bonds
// high-high), FP32 blocks of 8 with both walks in 128-thread CTAs: S^z = 0 / -5 /
// -6 / -7 (5, 0.96, 0.46, 0.19 GB) 16.7 -> 14.0, 3.18 -> 2.78, 1.54 -> 1.40, 0.669
// -> 0.661 ms; with walk A in blocks and 256-thread CTAs: FP32 blocks of 4 / 1 at
// S^z = 0 (2.5, 0.6 GB) 9.72 -> 9.22, 5.54 -> 6.15 ms, FP64 blocks of 4 (5 GB) 96.4
// -> 69.7 ms.  N = 34 ring (19 of 34 bonds high-high), FP32 blocks of 8, S^z = 0
// (75 GB): 177.1 -> 157.6 ms (179.0 -> 183.1 with 256-thread CTAs).  N = 26 ladder
// and ring (11 high-high bonds), S^z = 0, blocks of 8 (0.33 GB): 1.34 -> 1.41, 1.20
// -> 1.24 ms.  The split moves two row streams per step instead of one but no
// long-jump gather misses L2; with few high-high bonds per row, or on small blocks,
// the second pass costs more than the misses it saves.
constexpr uint64_t kSplitMinBytes32Rows = 256ull << 20;
constexpr uint64_t kSplitMinBytes32 = 768ull << 20;
constexpr uint64_t kSplitMinBytes64 = 1ull << 30;
constexpr int kSplitMinHiBonds = 16;
constexpr int kDefaultWalkRh = 8;

bool split_walks(const ftlm_basis *b, int B, size_t vsize, HiWalk *w)
{
    if (b->hv_schedule == FTLM_HV_ONE_WALK || !b->lo_tiles) return false;
    const uint64_t bytes = b->D * (uint64_t)B * vsize;
    const uint64_t min_bytes =
        vsize == 4 ? (B * vsize >= 32 ? kSplitMinBytes32Rows : kSplitMinBytes32) : kSplitMinBytes64;
    if (b->hv_schedule == FTLM_HV_AUTO && (bytes < min_bytes || b->n_hi_bonds < kSplitMinHiBonds)) return false;
    return build_hi_walk(b, b->walk_rh ? b->walk_rh : kDefaultWalkRh, w);
}

// One hv_kernel launch over every row.
template <typename V, typename Lbl, bool CLT, int EPI, int RT, int B, int C>
ftlm_status launch_rows(const ftlm_basis *b, const BondList &bl, const V *x, V *y, const EpiDev &ep,
                        cudaStream_t stream)
{
    const size_t smem = CLT ? 0 : ((size_t)1 << b->L) * sizeof(uint16_t);
    auto kern = hv_kernel<V, Lbl, CLT, EPI, RT, B, C>;
    int occ = 1;  // resident blocks per SM for this instantiation
    const size_t smem_max = CLT ? 0 : ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
    FTLM_CUDA(kernel_occupancy((const void *)kern, kRowThreads, smem_max, false, &occ));
    const int grid = row_grid(b, (b->D + RT - 1) / RT, std::min(occ, hv_cta_cap()));
    kern<<<grid, kRowThreads, smem, stream>>>(b->tables(), bl, x, y, ep);
    note_launch();
    return FTLM_OK;
}

// alpha_j from the per-tile sums of a dynamically ordered launch.
template <int B>
void launch_tile_alpha(const ftlm_basis *b, const EpiDev &ep, uint32_t ntiles, cudaStream_t stream)
{
    const int ga = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)b->num_sms * 2, (ntiles + 2047) / 2048));
    tile_alpha_kernel<B><<<ga, kRowThreads, 0, stream>>>(ep, ntiles);
    note_launch();
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS, int RT, int B, int C>
ftlm_status launch(const ftlm_basis *b, const V *x, V *y, const EpiDev &ep, cudaStream_t stream)
{
    void *tok = profile_begin(kProfHv, stream, B);
    ftlm_status st = FTLM_OK;
    if constexpr (LANCZOS && !CLT) {
        // CR Lanczos step: one walk over the rows, or the split (walk A, then walk B
        // over the high-high bonds in the transposed order); alpha_j from per-tile sums
        HiWalk w;
        uint32_t ntiles;
        if (split_walks(b, B, sizeof(V), &w)) {
            const ftlm_dtype dt = sizeof(V) == 4 ? FTLM_F32 : FTLM_F64;
            LoWalk la;
            st = build_lo_walk(b, &la) ? launch_walk_a(b, la, dt, B, x, y, ep, stream)
                                       : fail(FTLM_EUNSUPPORTED, "split H.v without a walk A tile table");
            if (st == FTLM_OK) st = launch_walk_b(b, w, dt, B, x, y, ep, stream);
            ntiles = w.ntiles;
        } else {
            st = launch_rows<V, Lbl, false, kLanczos, RT, B, C>(b, b->bonds_cr, x, y, ep, stream);
            const uint64_t rows = 32ull * RT;
            ntiles = (uint32_t)((b->D + rows - 1) / rows);
        }
        if (st == FTLM_OK) launch_tile_alpha<B>(b, ep, ntiles, stream);
    } else {
        st = launch_rows<V, Lbl, CLT, LANCZOS ? kLanczos : kPlain, RT, B, C>(b, CLT ? b->bonds_clt : b->bonds_cr, x,
                                                                           y, ep, stream);
    }
    profile_end(tok, stream);
    if (st != FTLM_OK) return st;
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

// Bonds per chunk for 8-wide blocks (FTLM_HV_CHUNK = 2, 4 or 8 overrides the
// default of 4): a larger chunk keeps more gathers in flight per row, a smaller
// one leaves registers for more resident warps.
int chunk8()
{
    static const int c = [] {
        const char *e = getenv("FTLM_HV_CHUNK");
        const int v = e ? atoi(e) : 0;
        return (v == 8 || v == 2) ? v : 4;
    }();
    return c;
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS>
ftlm_status launch_b(const ftlm_basis *b, int B, const void *x, void *y, const EpiDev &ep, cudaStream_t stream)
{
    const V *xv = (const V *)x;
    V *yv = (V *)y;
    switch (B) {
    case 4: return launch<V, Lbl, CLT, LANCZOS, 1, 4, 8>(b, xv, yv, ep, stream);
    case 8:
        switch (chunk8()) {
        case 8: return launch<V, Lbl, CLT, LANCZOS, 1, 8, 8>(b, xv, yv, ep, stream);
        case 2: return launch<V, Lbl, CLT, LANCZOS, 1, 8, 2>(b, xv, yv, ep, stream);
        default: return launch<V, Lbl, CLT, LANCZOS, 1, 8, 4>(b, xv, yv, ep, stream);
        }
    case 16: return launch<V, Lbl, CLT, LANCZOS, 1, 16, 4>(b, xv, yv, ep, stream);
    default: break;
    }
    switch (rows_per_thread(CLT)) {
    case 1: return launch<V, Lbl, CLT, LANCZOS, 1, 1, 8>(b, xv, yv, ep, stream);
    case 4: return launch<V, Lbl, CLT, LANCZOS, 4, 1, 8>(b, xv, yv, ep, stream);
    default: return launch<V, Lbl, CLT, LANCZOS, 2, 1, 8>(b, xv, yv, ep, stream);
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
    const EpiDev ep = epi_of(epi);
    if (epi) return launch_mode<V, true>(b, B, x, y, ep, stream);
    return launch_mode<V, false>(b, B, x, y, ep, stream);
}

}  // namespace

bool valid_block(int B) { return B == 1 || B == 4 || B == 8 || B == 16; }

uint32_t hv_lanczos_tiles(const ftlm_basis *b, int B)
{
    if (b->two_s > 1 || b->mode == FTLM_RANK_CLT) return 0;
    const uint64_t rows = 32ull * (B == 1 ? rows_per_thread(false) : 1);
    uint32_t n = (uint32_t)((b->D + rows - 1) / rows);
    HiWalk w;  // walk B has the most tiles with one high pattern per tile
    if (build_hi_walk(b, 1, &w)) n = std::max(n, w.ntiles);
    return n;
}

ftlm_status launch_hv(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y,
                      const LanczosHv *epi, cudaStream_t stream)
{
    if (b->two_s > 1) return launch_hv_spin(b, dtype, B, x, y, epi, stream);
    return dtype == FTLM_F32 ? launch_typed<float>(b, B, x, y, epi, stream)
                             : launch_typed<double>(b, B, x, y, epi, stream);
}

}  // namespace ftlm

namespace {
ftlm_status check_hv_args(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x_dev, void *y_dev)
{
    if (!b) return ftlm::fail(FTLM_EINVAL, "NULL basis");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return ftlm::fail(FTLM_EINVAL, "bad dtype");
    if (!x_dev || !y_dev) return ftlm::fail(FTLM_EINVAL, "NULL vector");
    if (x_dev == y_dev) return ftlm::fail(FTLM_EINVAL, "x and y must not overlap");
    // rows of 32 bytes or more move as 32-byte transactions
    const unsigned row = (unsigned)B * (dtype == FTLM_F32 ? 4u : 8u);
    const uintptr_t mask = row >= 32 ? 31u : 15u;
    if (((uintptr_t)x_dev | (uintptr_t)y_dev) & mask)
        return ftlm::fail(FTLM_EINVAL, row >= 32 ? "vectors must be 32-byte aligned for rows of 32 bytes or more"
                                                 : "vectors must be 16-byte aligned");
    return FTLM_OK;
}
}  // namespace

extern "C" ftlm_status ftlm_basis_hv_schedule(const ftlm_basis *b, int B, ftlm_dtype dtype, ftlm_hv_schedule *used)
{
    if (!b || !used) return ftlm::fail(FTLM_EINVAL, "NULL argument");
    if (!ftlm::valid_block(B)) return ftlm::fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return ftlm::fail(FTLM_EINVAL, "bad dtype");
    ftlm::HiWalk w;
    const bool split = b->two_s == 1 && b->mode == FTLM_RANK_CR &&
                       ftlm::split_walks(b, B, dtype == FTLM_F32 ? 4 : 8, &w);
    *used = split ? FTLM_HV_SPLIT : FTLM_HV_ONE_WALK;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_hv(const ftlm_basis *b, ftlm_dtype dtype, const void *x_dev, void *y_dev,
                               void *stream)
{
    ftlm_status s = check_hv_args(b, dtype, 1, x_dev, y_dev);
    if (s != FTLM_OK) return s;
    return ftlm::launch_hv(b, dtype, 1, x_dev, y_dev, nullptr, (cudaStream_t)stream);
}

extern "C" ftlm_status ftlm_hv_block(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x_dev,
                                     void *y_dev, void *stream)
{
    if (!ftlm::valid_block(B)) return ftlm::fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    ftlm_status s = check_hv_args(b, dtype, B, x_dev, y_dev);
    if (s != FTLM_OK) return s;
    return ftlm::launch_hv(b, dtype, B, x_dev, y_dev, nullptr, (cudaStream_t)stream);
}
