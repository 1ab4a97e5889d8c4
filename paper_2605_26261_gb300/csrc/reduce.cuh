// Deterministic FP64 reductions for the row-parallel kernels.
//
// Each block reduces its per-thread partial sums in a fixed tree (warp shuffle,
// then one warp over the per-warp sums) and stores one partial per block.  The
// last block to finish -- found with a fence and an atomic ticket, no waiting --
// adds the per-block partials in index order and publishes the total.  For a
// fixed grid the summation order never changes, so results are bit-reproducible.
#pragma once

#include "ftlm_internal.cuh"

namespace ftlm {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;  // use lane 0's value: lanes may differ in the last bit
}

// Sum over the block; the result is valid in thread 0.
template <int THREADS>
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (lane < THREADS / 32) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Publish this block's partial; returns true (in every thread) in the last block
// of the grid to arrive.
__device__ __forceinline__ bool publish_partial(double part, double *partials, unsigned int *counter)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = part;
        __threadfence();
        unsigned int ticket = atomicAdd(counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    return last;
}

// Fixed-order total of partials[0 .. n-1]; call from warp 0, valid in lane 0.
__device__ __forceinline__ double total_of_partials(const double *partials, int n)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < n; i += 32) v += __ldcg(partials + i);
    return warp_sum(v);
}

}  // namespace ftlm

namespace ftlm {

// Per-thread accumulator of dot-product terms a * b.  For FP32 operands every
// product is split exactly into p + e (p = fl(a b), e = fma(a, b, -p)) and added
// to a two-float sum (hi, lo) with the error-free TwoSum of Knuth, so the running
// sum keeps about 48 significant bits without touching the FP64 pipe, which is
// narrow on GB300; value() hands the sum to the FP64 block and grid reductions.
// FP64 operands accumulate in FP64 directly.
template <typename V> struct DotAcc;

template <> struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    // The _rn intrinsics are never contracted into FMAs: TwoSum needs the rounded
    // product p, not a fused hi + a * b.
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bv = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    // Adds another accumulator: TwoSum of the high parts, low parts summed.  The
    // TwoSum error is exact, so a.merge(b) and b.merge(a) give the same bits.
    __device__ __forceinline__ void merge(const DotAcc &o)
    {
        const float s = __fadd_rn(hi, o.hi);
        const float bv = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(o.hi, bv));
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, o.lo), err);
    }
    __device__ __forceinline__ DotAcc shfl_xor(int o) const
    {
        DotAcc r;
        r.hi = __shfl_xor_sync(0xffffffffu, hi, o);
        r.lo = __shfl_xor_sync(0xffffffffu, lo, o);
        return r;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <> struct DotAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ void merge(const DotAcc &o) { v += o.v; }
    __device__ __forceinline__ DotAcc shfl_xor(int o) const
    {
        DotAcc r;
        r.v = __shfl_xor_sync(0xffffffffu, v, o);
        return r;
    }
    __device__ __forceinline__ double value() const { return v; }
};

// Warp sums of B accumulators (B = 1, 2, 4, 8 or 16) by a transposed butterfly: at
// each of the first log2(B) levels a lane keeps one half of its partial sums, sends
// the other half to its partner and merges what it receives (B - 1 merges and
// shuffles in all, instead of 5 B), then a plain butterfly over the remaining
// lanes.  Lane l ends with the sum of accumulator warp_multi_index<B>(l): the bit
// reversal of its low log2(B) bits, so lanes 0 .. B-1 hold the B sums.  The tree
// is fixed: reproducible.
template <typename V, int B>
__device__ __forceinline__ DotAcc<V> warp_sum_multi(DotAcc<V> (&a)[B])
{
    static_assert(B == 1 || B == 2 || B == 4 || B == 8 || B == 16, "B must be a power of two <= 16");
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int lvl = 0; (B >> lvl) > 1; ++lvl) {
        const int h = (B >> lvl) / 2;
        const bool upper = (lane >> lvl) & 1u;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            DotAcc<V> keep = upper ? a[i + h] : a[i];
            const DotAcc<V> send = upper ? a[i] : a[i + h];
            keep.merge(send.shfl_xor(1 << lvl));
            a[i] = keep;
        }
    }
    DotAcc<V> t = a[0];
#pragma unroll
    for (int o = B; o < 32; o <<= 1) t.merge(t.shfl_xor(o));
    return t;
}

template <int B> __device__ __forceinline__ int warp_multi_index(unsigned lane)
{
    int r = 0;
#pragma unroll
    for (int lvl = 0; (B >> lvl) > 1; ++lvl) r += ((lane >> lvl) & 1u) ? (B >> (lvl + 1)) : 0;
    return r;
}

}  // namespace ftlm
