// Lanczos epilogue of the H.v launches (step a4 fused into step a3), shared by the
// spin-1/2 kernel (hv.cu) and the general-spin kernel (spin.cu).
//
// Paige's ordering, per chain r of a block of B interleaved vectors.  The stored
// vector u_j is un-normalized, q_j = u_j / s_j.  With x = u_j and the in-place
// buffer holding u_{j-1}:
//   y[t] = (H u_j)[t] / s_j - (beta_{j-1} / s_{j-1}) u_{j-1}[t]     (overwrites u_{j-1})
//   alpha partial += q_j[t] y[t]                                    (FP64-class)
// Per-thread partial dot products use DotAcc (exact products, two-float
// compensated sums for FP32 vectors).  Two ways to finish alpha_j:
//  - static tile order (a warp takes every nwarps-th tile of rows): the block sum
//    is an FP64 tree and the last block to finish adds the per-block partials in
//    a fixed order and stores alpha_j (epi_end);
//  - dynamic tile order (CR launches: tiles handed out by a counter, so that all
//    warps work on one frontier of rows and the gathers of the rows in flight
//    share L2): each tile's sums go through a fixed warp tree into a slot of their
//    own (store_tile), and a second launch adds the slots in tile order.
// Both orders are fixed for a given sector and grid: alpha_j is reproducible.
#pragma once

#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "vec.cuh"

namespace ftlm {

struct EpiDev {
    ChainState *st;
    double *partials;
    unsigned int *counter;  // [0] block ticket; [1], [2] dynamic tile order
    double *alpha_out;
    double *tile_part;      // per-tile sums of the dynamic tile order, [tile][B]
    int alpha_stride;
    int has_prev;
};

inline EpiDev epi_of(const LanczosHv *epi)
{
    EpiDev ep{};
    if (epi) {
        ep.st = epi->st;
        ep.partials = epi->partials;
        ep.counter = epi->counter;
        ep.alpha_out = epi->alpha_out;
        ep.tile_part = epi->tile_part;
        ep.alpha_stride = epi->alpha_stride;
        ep.has_prev = epi->j > 1;
    }
    return ep;
}

// Per-chain scalars 1/s_j and beta_{j-1}/s_{j-1} into shared memory.  Returns true
// (in every thread) when every chain of the block has stopped: the launch then has
// nothing to do, and the test is uniform over the grid.
template <typename V, int B>
__device__ __forceinline__ bool epi_begin(const EpiDev &ep, V *s_inv_s, V *s_c_prev)
{
    bool all_stopped = true;
#pragma unroll
    for (int r = 0; r < B; ++r) all_stopped &= ep.st[r].stopped != 0;
    if (all_stopped) return true;
    if (threadIdx.x < B) {
        const ChainState &st = ep.st[threadIdx.x];
        s_inv_s[threadIdx.x] = (V)(1.0 / st.s_cur);
        s_c_prev[threadIdx.x] = ep.has_prev ? (V)(st.beta_prev / st.s_prev) : (V)0;
    }
    return false;
}

// Output row t: y = diag * x[t] + acc (plain H.v) or the epilogue above.
template <typename V, int B, bool LANCZOS>
__device__ __forceinline__ void epi_row(const EpiDev &ep, const V *s_inv_s, const V *s_c_prev,
                                        const V *__restrict__ x, V *y, uint32_t t, V diag, const V (&acc)[B],
                                        DotAcc<V> (&apart)[B])
{
    V xt[B], out[B];
    ld_vec<B>(x + (size_t)t * B, xt, false);
    if (LANCZOS) {
        V up[B];
        if (ep.has_prev) ld_vec<B>(y + (size_t)t * B, up, true);
#pragma unroll
        for (int r = 0; r < B; ++r) {
            const V inv_s = s_inv_s[r];
            const V hv = fma(diag, xt[r], acc[r]);
            out[r] = ep.has_prev ? fma(-s_c_prev[r], up[r], hv * inv_s) : hv * inv_s;
            apart[r].add(xt[r] * inv_s, out[r]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < B; ++r) out[r] = fma(diag, xt[r], acc[r]);
    }
    st_vec<B>(y + (size_t)t * B, out);
}

// Output row t of walk A of a split H.v (CR): the Lanczos output of the bonds of
// walk A, y = (H_A u_j)[t] / s_j - (beta_{j-1} / s_{j-1}) u_{j-1}[t], with no alpha
// partial (walk B adds the rest of the row and finishes alpha).
template <typename V, int B>
__device__ __forceinline__ void epi_row_walk_a(const EpiDev &ep, const V *s_inv_s, const V *s_c_prev,
                                               const V *__restrict__ x, V *y, uint32_t t, V diag,
                                               const V (&acc)[B])
{
    V xt[B], out[B], up[B];
    ld_vec<B>(x + (size_t)t * B, xt, false);
    if (ep.has_prev) ld_vec<B>(y + (size_t)t * B, up, true);
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const V hv = fma(diag, xt[r], acc[r]);
        out[r] = ep.has_prev ? fma(-s_c_prev[r], up[r], hv * s_inv_s[r]) : hv * s_inv_s[r];
    }
    st_vec<B>(y + (size_t)t * B, out);
}

// Block sums of the alpha partials, publication, and the last block's fixed-order
// grid sum into alpha_j (chains that have stopped keep their value).
template <typename V, int B, int THREADS>
__device__ __forceinline__ void epi_end(const EpiDev &ep, DotAcc<V> (&apart)[B])
{
    __shared__ double s_part[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const double part = block_sum<THREADS>(apart[r].value());
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

// Dynamic tile order: a warp's first tile is its index, later ones come from the
// counter ep.counter[1]; ep.counter[2] counts the warps that ran out of tiles, and
// the last of them zeroes both for the next launch (they start at zero).  A warp
// claims its next tile when it starts a tile (claim_tile, lane 0) and reads the
// claim when it finishes (claimed_tile), so the atomic's round trip is hidden.
__device__ __forceinline__ uint32_t claim_tile(const EpiDev &ep)
{
    return (threadIdx.x & 31u) == 0 ? atomicAdd(ep.counter + 1, 1u) : 0u;
}

__device__ __forceinline__ uint32_t claimed_tile(uint32_t claim, uint32_t nwarps)
{
    return __shfl_sync(0xffffffffu, claim, 0) + nwarps;
}

__device__ __forceinline__ void tiles_done(const EpiDev &ep, uint32_t nwarps)
{
    if ((threadIdx.x & 31u) == 0) {
        __threadfence();
        if (atomicAdd(ep.counter + 2, 1u) == nwarps - 1) {
            ep.counter[1] = 0;
            ep.counter[2] = 0;
        }
    }
}

// The warp's alpha partial sums of one tile, through a fixed warp tree, into
// ep.tile_part[tile * B + r].  Called by the whole warp.
template <typename V, int B>
__device__ __forceinline__ void store_tile(const EpiDev &ep, uint32_t tile, DotAcc<V> (&a)[B])
{
    const DotAcc<V> t = warp_sum_multi<V, B>(a);
    const unsigned lane = threadIdx.x & 31u;
    if (lane < B) ep.tile_part[(size_t)tile * B + warp_multi_index<B>(lane)] = t.value();
}

}  // namespace ftlm
