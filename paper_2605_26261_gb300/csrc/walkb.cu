// Walk B of the split Lanczos H.v (CR, spin 1/2): the high-high bonds of Eq. 12-14
// in the transposed row order, added to walk A's output, with the Lanczos epilogue
// (alpha as per-tile sums).  The layout of the walk is described with HiWalk in
// ftlm_internal.cuh.
//
// A warp owns a tile: 32 consecutive low ranks r_lo (lane = column) of one low
// popcount group q, and a run of rh high patterns h of popcount K - q.  Row (h, l)
// sits at thi[h] + r_lo, so for each h the warp's 32 rows are contiguous.  A
// high-high bond m leaves l alone: the source row is thi[h ^ m] + r_lo, again 32
// contiguous rows, and whether the bond is antiparallel depends on h only, which
// is the same in every lane.  Per h the lanes test the bonds in parallel (lane b
// holds bond b and looks up thi[h ^ m_b]); a ballot gives the antiparallel set, and
// the warp then walks it uniformly, without predication, in chunks of C bonds whose
// gathers are all issued before the first one is used.  Only the rank r_lo of l
// within its popcount group enters, never l itself, so walk B needs no low-block
// table at all.
//
// Rows per lane: one per high pattern of the tile.  Per row the walk reads walk A's
// partial output y[t] and x[t] (for the diagonal part of the high-high bonds and
// for alpha) and writes y[t] once.
#include <algorithm>

#include "epi.cuh"
#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "vec.cuh"

namespace ftlm {

namespace {

template <typename V> __device__ __forceinline__ V hi_jh(const uint4 &e);
template <> __device__ __forceinline__ float hi_jh<float>(const uint4 &e) { return __uint_as_float(e.y); }
template <> __device__ __forceinline__ double hi_jh<double>(const uint4 &e)
{
    return __hiloint2double((int)e.w, (int)e.z);
}

// CTA size and resident CTAs per SM the register budget allows for: walk B keeps C
// gathered rows of B values and the row's own two rows in flight per lane.  Rows of
// 32 bytes run in CTAs of 128 threads, 5 per SM (96 registers): 20 warps per SM
// against 16 in 256-thread CTAs at 116 registers, 14.98 against 15.80 ms per H.v
// step on the N = 30 sector (FP32 blocks of 8).
template <typename V, int B> __host__ __device__ constexpr int walk_b_threads()
{
    return sizeof(V) * B == 32 ? 128 : kRowThreads;
}
template <typename V, int B> __host__ __device__ constexpr int walk_b_min_ctas()
{
    return sizeof(V) * B >= 64 ? 1 : (sizeof(V) * B >= 32 ? 5 : (sizeof(V) * B >= 8 ? 3 : 4));
}

template <typename V, int B, int C>
__global__ void __launch_bounds__(walk_b_threads<V, B>(), walk_b_min_ctas<V, B>())
walk_b_kernel(const uint32_t *__restrict__ thi, const HiWalk w, const V *__restrict__ x, V *y, const EpiDev ep)
{
    __shared__ V s_inv_s[B], s_c_prev[B];
    __shared__ uint32_t s_tile0[kMaxHiGroups + 1], s_nl[kMaxHiGroups], s_nh[kMaxHiGroups],
        s_hoff[kMaxHiGroups], s_nr[kMaxHiGroups];
    if (epi_begin<V, B>(ep, s_inv_s, s_c_prev)) return;
    // group tables into shared memory (a kernel-parameter array indexed at run time
    // would be copied to local memory)
    if (threadIdx.x <= (unsigned)w.ngroups) s_tile0[threadIdx.x] = w.tile0[threadIdx.x];
    if (threadIdx.x < (unsigned)w.ngroups) {
        s_nl[threadIdx.x] = w.nl[threadIdx.x];
        s_nh[threadIdx.x] = w.nh[threadIdx.x];
        s_hoff[threadIdx.x] = w.hoff[threadIdx.x];
        s_nr[threadIdx.x] = w.nr[threadIdx.x];
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    // bond lane and lane + 32 of the walk: high-block mask and J/2 (mask 0: none)
    uint32_t bm[2];
    V bj[2];
#pragma unroll
    for (int wd = 0; wd < 2; ++wd) {
        const int k = (int)lane + 32 * wd;
        if (k < w.nbonds) {
            const uint4 e = w.bonds[k];
            bm[wd] = e.x;
            bj[wd] = hi_jh<V>(e);
        } else {
            bm[wd] = 0u;
            bj[wd] = (V)0;
        }
    }
    const V jsum4 = (V)w.jsum4;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t rh = (uint32_t)w.rh;

    for (uint32_t tile = warp; tile < w.ntiles;) {
        const uint32_t claim = claim_tile(ep);
        int g = 0;
        while (g + 1 < w.ngroups && tile >= s_tile0[g + 1]) ++g;
        const uint32_t rel = tile - s_tile0[g];
        const uint32_t nr = s_nr[g];
        const uint32_t chunk = rel / nr, run = rel - chunk * nr;
        const uint32_t li = chunk * 32u + lane;
        const bool valid = li < s_nl[g];
        const uint32_t k0 = run * rh;
        const uint32_t kn = min(s_nh[g], k0 + rh) - k0;  // high patterns of the tile (<= 32)
        // the tile's high patterns and their row bases, one per lane
        const uint32_t h_l = lane < kn ? __ldg(w.uhi + s_hoff[g] + k0 + lane) : 0u;
        const uint32_t rb_l = lane < kn ? __ldg(thi + h_l) : 0u;
        DotAcc<V> tacc[B];
        for (uint32_t k = 0; k < kn; ++k) {
            const uint32_t h = __shfl_sync(0xffffffffu, h_l, k);
            const uint32_t rb = __shfl_sync(0xffffffffu, rb_l, k);
            // the row's own entries first: their DRAM latency overlaps the gathers
            const size_t t = (size_t)(rb + li);
            V xt[B], yv[B];
            if (valid) {
                ld_vec<B>(x + t * B, xt, false);
                ld_vec<B>(y + t * B, yv, true);
            }
            uint32_t amask[2], src[2];
#pragma unroll
            for (int wd = 0; wd < 2; ++wd) {
                const uint32_t xm = h & bm[wd];
                const bool anti = (xm != 0u) & (xm != bm[wd]);
                src[wd] = anti ? __ldg(thi + (h ^ bm[wd])) : 0u;
                amask[wd] = __ballot_sync(0xffffffffu, anti);
            }
            V acc[B];
#pragma unroll
            for (int r = 0; r < B; ++r) acc[r] = (V)0;
            V dsum = (V)0;
#pragma unroll
            for (int wd = 0; wd < 2; ++wd) {  // the second word is empty for <= 32 bonds
                uint32_t mk = amask[wd];
                while (mk) {  // uniform over the warp
                    V xv[C][B], jq[C];
#pragma unroll
                    for (int q = 0; q < C; ++q) {
                        const bool on = mk != 0u;
                        const int bit = on ? __ffs(mk) - 1 : 0;
                        mk &= mk - 1u;
                        const uint32_t sq = __shfl_sync(0xffffffffu, src[wd], bit);
                        const V jb = __shfl_sync(0xffffffffu, bj[wd], bit);
                        jq[q] = on ? jb : (V)0;
                        if (on && valid) {
                            ld_vec<B>(x + (size_t)(sq + li) * B, xv[q], false);
                        } else {
#pragma unroll
                            for (int r = 0; r < B; ++r) xv[q][r] = (V)0;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < C; ++q) {
#pragma unroll
                        for (int r = 0; r < B; ++r) acc[r] = fma(jq[q], xv[q][r], acc[r]);
                        dsum += jq[q];
                    }
                }
            }
            if (valid) {
                V out[B];
                const V diag = jsum4 - dsum;
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    out[r] = fma(fma(diag, xt[r], acc[r]), s_inv_s[r], yv[r]);
                    tacc[r].add(xt[r] * s_inv_s[r], out[r]);
                }
                st_vec<B>(y + t * B, out);
            }
        }
        store_tile<V, B>(ep, tile, tacc);
        tile = claimed_tile(claim, nwarps);
    }
    tiles_done(ep, nwarps);
}

template <typename V, int B, int C>
ftlm_status launch_typed(const ftlm_basis *b, const HiWalk &w, const V *x, V *y, const EpiDev &ep,
                         cudaStream_t stream)
{
    auto kern = walk_b_kernel<V, B, C>;
    constexpr int T = walk_b_threads<V, B>();
    int occ = 1;
    FTLM_CUDA(kernel_occupancy((const void *)kern, T, 0, false, &occ));
    const uint64_t need = ((uint64_t)w.ntiles * 32 + T - 1) / T;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)b->num_sms * occ));
    kern<<<grid, T, 0, stream>>>(b->thi, w, x, y, ep);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V>
ftlm_status launch_width(const ftlm_basis *b, const HiWalk &w, int B, const void *x, void *y, const EpiDev &ep,
                         cudaStream_t stream)
{
    const V *xv = (const V *)x;
    V *yv = (V *)y;
    switch (B) {
    case 16: return launch_typed<V, 16, 2>(b, w, xv, yv, ep, stream);
    case 8: return launch_typed<V, 8, 4>(b, w, xv, yv, ep, stream);
    case 4: return launch_typed<V, 4, 4>(b, w, xv, yv, ep, stream);
    case 1: return launch_typed<V, 1, 8>(b, w, xv, yv, ep, stream);
    default: return fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    }
}

}  // namespace

ftlm_status launch_walk_b(const ftlm_basis *b, const HiWalk &w, ftlm_dtype dtype, int B, const void *x, void *y,
                          const EpiDev &ep, cudaStream_t stream)
{
    if (w.ntiles == 0) return FTLM_OK;
    return dtype == FTLM_F32 ? launch_width<float>(b, w, B, x, y, ep, stream)
                             : launch_width<double>(b, w, B, x, y, ep, stream);
}

}  // namespace ftlm
