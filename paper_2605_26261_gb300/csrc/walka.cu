// Walk A of the split Lanczos H.v (CR, spin 1/2) in blocks: the lo-lo and cross
// bonds of Eq. 12-14, with the Lanczos epilogue that walk B completes.  The tile
// layout is described with LoWalk in ftlm_internal.cuh.
//
// A warp owns a tile: 32 consecutive low ranks (lane = column, low pattern l of
// popcount q, one ulo lookup per tile) and a run of up to kLoRun high patterns h of
// popcount K - q (lanes 0 .. kLoRun-1 look up h and its row base thi[h], then
// shuffle).  It takes the run's rows RH at a time (RH high patterns x 32 columns):
//   lo-lo bonds   antiparallel or not and the source rank tlo[l ^ m] depend on l
//                 only: one shared-memory lookup per bond serves the RH rows, whose
//                 gathers (thi[h_k] + tlo[l ^ m]) are issued together;
//   cross bonds   the low half tlo[l ^ 2^i] is per lane, the high half
//                 thi[h_k ^ 2^(j-L)] the same in every lane (one broadcast load);
// then each row is written once as (H_A u_j)[t] / s_j - (beta_{j-1}/s_{j-1})
// u_{j-1}[t] (epi_row_walk_a), t = thi[h_k] + 32 c + lane.  Against the walk in
// label order (one row per lane, its label recovered by a search of thi and a
// lookup of ulo, then one tlo lookup per bond and row) this takes the per-row
// inverse map out and divides the shared-memory lookups -- whose scattered
// addresses cost about 2.8 wavefronts each through bank conflicts -- by RH.
#include <algorithm>
#include <cstdlib>

#include "epi.cuh"
#include "ftlm_internal.cuh"
#include "rows.cuh"
#include "vec.cuh"

namespace ftlm {

namespace {

// High patterns per pass: RH x B accumulators and as many gathers in flight.
template <typename V, int B> __host__ __device__ constexpr int walk_a_rows()
{
    return (int)sizeof(V) * B <= 32 ? 4 : ((int)sizeof(V) * B <= 64 ? 2 : 1);
}

// CTA size and resident CTAs per SM the register budget allows for: RH x B
// accumulators and as many gathered values in flight per lane.  FP32 blocks of 8
// with 4 high patterns per pass run in CTAs of 128 threads, 5 per SM (96 registers,
// no spills): 20 warps per SM against 16 in 256-thread CTAs at 103 registers.
template <typename V, int B, int RH> __host__ __device__ constexpr int walk_a_threads()
{
    return (sizeof(V) == 4 && B == 8 && RH == 4) ? 128 : kRowThreads;
}
template <typename V, int B, int RH> __host__ __device__ constexpr int walk_a_min_ctas()
{
    return walk_a_threads<V, B, RH>() == 128
               ? 5
               : (RH * B * (int)sizeof(V) >= 128 ? 2 : (RH * B * (int)sizeof(V) >= 64 ? 3 : 4));
}

template <typename V, int B, int RH>
__global__ void __launch_bounds__(walk_a_threads<V, B, RH>(), walk_a_min_ctas<V, B, RH>())
walk_a_kernel(const SectorTables s, const LoWalk w, const V *__restrict__ x, V *y, const EpiDev ep)
{
    extern __shared__ uint16_t s_tlo[];
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ V s_inv_s[B], s_c_prev[B];
    __shared__ uint32_t s_uoff[kLoBitsMax + 2], s_hend[kMaxHighBits + 2];
    if (epi_begin<V, B>(ep, s_inv_s, s_c_prev)) return;
    {
        const uint4 *src = sizeof(V) == 4 ? w.slots_f32 : w.slots_f64;
        for (int i = threadIdx.x; i < w.nb; i += blockDim.x) s_bond[i] = src[i];
    }
    for (uint32_t i = threadIdx.x; i <= s.lomask; i += blockDim.x) s_tlo[i] = __ldg(s.tlo + i);
    if (threadIdx.x < kLoBitsMax + 2) s_uoff[threadIdx.x] = __ldg(s.uoff + threadIdx.x);
    if (threadIdx.x < kMaxHighBits + 2) s_hend[threadIdx.x] = w.hend[threadIdx.x];
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const V jsum4 = (V)w.jsum4;
    const int e_ll = w.n_ll, e_all = w.n_ll + w.n_cr;

    for (uint32_t tile = warp; tile < w.ntiles;) {
        // claim the next tile now; its atomic completes while this tile's rows run
        const uint32_t claim = claim_tile(ep);
        const uint32_t e = __ldg(w.tiles + tile);
        const uint32_t pos = e >> 7, chunk = e & 127u;
        const uint32_t p = (uint32_t)__popc(__ldg(w.uhi + pos));
        const uint32_t q = (uint32_t)s.K - p;  // a valid low popcount by construction
        const uint32_t kn = min((uint32_t)kLoRun, s_hend[p] - pos);
        const uint32_t h_l = lane < kn ? __ldg(w.uhi + pos + lane) : 0u;
        const uint32_t rb_l = lane < kn ? __ldg(s.thi + h_l) : 0u;
        const uint32_t li = chunk * 32u + lane;
        const bool valid = li < s_uoff[q + 1] - s_uoff[q];
        const uint32_t l = valid ? (uint32_t)__ldg(s.ulo + s_uoff[q] + li) : 0u;
#pragma unroll
        for (uint32_t k0 = 0; k0 < (uint32_t)kLoRun; k0 += RH) {
            if (k0 >= kn) break;  // uniform over the warp
            uint32_t hk[RH], rbk[RH];
            bool ok[RH];
#pragma unroll
            for (int i = 0; i < RH; ++i) {
                ok[i] = valid && (k0 + i < kn);
                hk[i] = __shfl_sync(0xffffffffu, h_l, k0 + i);
                rbk[i] = __shfl_sync(0xffffffffu, rb_l, k0 + i);
            }
            V acc[RH][B], dcr[RH], dll = (V)0;
#pragma unroll
            for (int i = 0; i < RH; ++i) {
                dcr[i] = (V)0;
#pragma unroll
                for (int r = 0; r < B; ++r) acc[i][r] = (V)0;
            }
            // lo-lo bonds: one rank per bond for the RH rows; the next bond's rank is
            // looked up one bond ahead
            uint32_t src_n = 0u;
            bool anti_n = false;
            V jh_n = (V)0;
            auto look = [&](int b) {
                const uint4 eb = s_bond[b];  // same address in every lane: a broadcast
                const uint32_t m = eb.x, xm = l & m;
                anti_n = valid && (xm != 0u) && (xm != m);
                jh_n = slot_jh<V>(eb);
                src_n = anti_n ? (uint32_t)s_tlo[l ^ m] : 0u;
            };
            if (e_ll > 0) look(0);
            for (int b = 0; b < e_ll; ++b) {
                const uint32_t src = src_n;
                const bool anti = anti_n;
                const V jh = jh_n;
                if (b + 1 < e_ll) look(b + 1);
                V xv[RH][B];
#pragma unroll
                for (int i = 0; i < RH; ++i) {
                    if (anti && ok[i]) {
                        ld_vec<B>(x + (size_t)(rbk[i] + src) * B, xv[i], false);
                    } else {
#pragma unroll
                        for (int r = 0; r < B; ++r) xv[i][r] = (V)0;
                    }
                }
                if (anti) {
#pragma unroll
                    for (int i = 0; i < RH; ++i)
#pragma unroll
                        for (int r = 0; r < B; ++r) acc[i][r] = fma(jh, xv[i][r], acc[i][r]);
                    dll += jh;
                }
            }
            // cross bonds: per-lane low half, warp-uniform high half per row
            for (int b = e_ll; b < e_all; ++b) {
                const uint4 eb = s_bond[b];
                const uint32_t ml = eb.x, mh = eb.y;
                const V jh = slot_jh<V>(eb);
                const bool lbit = (l & ml) != 0u;
                const uint32_t lt = (valid && ml) ? (uint32_t)s_tlo[l ^ ml] : 0u;
                bool an[RH];
                V xv[RH][B];
#pragma unroll
                for (int i = 0; i < RH; ++i) {
                    an[i] = ok[i] && ml != 0u && (lbit != ((hk[i] & mh) != 0u));
                    if (an[i]) {
                        const uint32_t src = __ldg(s.thi + (hk[i] ^ mh)) + lt;
                        ld_vec<B>(x + (size_t)src * B, xv[i], false);
                    } else {
#pragma unroll
                        for (int r = 0; r < B; ++r) xv[i][r] = (V)0;
                    }
                }
#pragma unroll
                for (int i = 0; i < RH; ++i)
                    if (an[i]) {
#pragma unroll
                        for (int r = 0; r < B; ++r) acc[i][r] = fma(jh, xv[i][r], acc[i][r]);
                        dcr[i] += jh;
                    }
            }
#pragma unroll
            for (int i = 0; i < RH; ++i)
                if (ok[i])
                    epi_row_walk_a<V, B>(ep, s_inv_s, s_c_prev, x, y, rbk[i] + li, jsum4 - dll - dcr[i], acc[i]);
        }
        tile = claimed_tile(claim, nwarps);
    }
    tiles_done(ep, nwarps);
}

// High patterns per pass (FTLM_WALKA_RH = 1, 2 or 4 lowers the default).
int walk_a_rh(int dflt)
{
    static const int v = [] {
        const char *e = getenv("FTLM_WALKA_RH");
        const int r = e ? atoi(e) : 0;
        return (r == 1 || r == 2 || r == 4) ? r : 0;
    }();
    return v ? std::min(v, dflt) : dflt;
}

template <typename V, int B, int RH>
ftlm_status launch_rh(const ftlm_basis *b, const LoWalk &w, const V *x, V *y, const EpiDev &ep,
                      cudaStream_t stream)
{
    auto kern = walk_a_kernel<V, B, RH>;
    const size_t smem = ((size_t)1 << b->L) * sizeof(uint16_t);
    const size_t smem_max = ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
    int occ = 1;
    constexpr int T = walk_a_threads<V, B, RH>();
    FTLM_CUDA(kernel_occupancy((const void *)kern, T, smem_max, false, &occ));
    const uint64_t need = ((uint64_t)w.ntiles * 32 + T - 1) / T;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)b->num_sms * occ));
    kern<<<grid, T, smem, stream>>>(b->tables(), w, x, y, ep);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V, int B>
ftlm_status launch_typed(const ftlm_basis *b, const LoWalk &w, const V *x, V *y, const EpiDev &ep,
                         cudaStream_t stream)
{
    constexpr int RH = walk_a_rows<V, B>();
    switch (walk_a_rh(RH)) {
    case 1: return launch_rh<V, B, 1>(b, w, x, y, ep, stream);
    case 2: return launch_rh<V, B, (RH >= 2 ? 2 : 1)>(b, w, x, y, ep, stream);
    default: return launch_rh<V, B, RH>(b, w, x, y, ep, stream);
    }
}

template <typename V>
ftlm_status launch_width(const ftlm_basis *b, const LoWalk &w, int B, const void *x, void *y, const EpiDev &ep,
                         cudaStream_t stream)
{
    const V *xv = (const V *)x;
    V *yv = (V *)y;
    switch (B) {
    case 16: return launch_typed<V, 16>(b, w, xv, yv, ep, stream);
    case 8: return launch_typed<V, 8>(b, w, xv, yv, ep, stream);
    case 4: return launch_typed<V, 4>(b, w, xv, yv, ep, stream);
    case 1: return launch_typed<V, 1>(b, w, xv, yv, ep, stream);
    default: return fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    }
}

}  // namespace

ftlm_status launch_walk_a(const ftlm_basis *b, const LoWalk &w, ftlm_dtype dtype, int B, const void *x, void *y,
                          const EpiDev &ep, cudaStream_t stream)
{
    if (w.ntiles == 0) return FTLM_OK;
    return dtype == FTLM_F32 ? launch_width<float>(b, w, B, x, y, ep, stream)
                             : launch_width<double>(b, w, B, x, y, ep, stream);
}

}  // namespace ftlm
