// Row work of the H.v gather (Eq. 12-14 at s = 1/2) shared by the single-launch
// kernel (hv.cu) and the batched kernel (batch.cu): the inverse map of a row, the
// rank of every exchanged label (CR digit blocks or CLT), and the chunked,
// predicated gathers of B interleaved vectors.  NC = true gathers through the
// read-only path (x is not written during the launch); the batched kernel, which
// rewrites its vectors between passes, uses coherent loads.
#pragma once

#include "ftlm_internal.cuh"
#include "vec.cuh"

namespace ftlm {

// J/2 of a bond slot in the vector type.
template <typename V> __device__ __forceinline__ V slot_jh(const uint4 &e);
template <> __device__ __forceinline__ float slot_jh<float>(const uint4 &e) { return __uint_as_float(e.z); }
template <> __device__ __forceinline__ double slot_jh<double>(const uint4 &e)
{
    return __hiloint2double((int)e.w, (int)e.z);
}


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
template <typename V, int RT, int B, int C, bool NC = true>
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
                if constexpr (NC) ld_vec<B>(x + (size_t)kk[i][q] * B, xv[i][q], false);
                else ld_vec_coherent<B>(x + (size_t)kk[i][q] * B, xv[i][q]);
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
template <typename V, typename Lbl, int RT, int B, int C, bool NC = true>
__device__ __forceinline__ void rows_cr(const SectorTables &s, const BondList &bl, const uint4 *s_bond,
                                        const uint16_t *s_tlo, const V *__restrict__ x,
                                        const uint32_t (&t)[RT], V (&acc)[RT][B], V (&dsum)[RT])
{
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
        gather_accumulate<V, RT, B, C, NC>(x, c, aa, kk, acc, dsum);
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
        gather_accumulate<V, RT, B, C, NC>(x, c, aa, kk, acc, dsum);
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
        gather_accumulate<V, RT, B, C, NC>(x, c, aa, kk, acc, dsum);
    }
}

// Row sums of RT output rows (CLT, Algorithm 2 per exchanged label).
template <typename V, int RT, int B, int C, bool NC = true>
__device__ __forceinline__ void rows_clt(const SectorTables &s, const BondList &bl, const uint4 *s_bond,
                                         const V *__restrict__ x, const uint32_t (&t)[RT], V (&acc)[RT][B],
                                         V (&dsum)[RT])
{
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
        gather_accumulate<V, RT, B, C, NC>(x, c, aa, kk, acc, dsum);
    }
}

// One warp owns a tile of 32 RT consecutive rows; lane l handles rows
// tile_base + l + 32 i (i < RT).  The launches hand the tiles out in row order --
// round-robin over the warps (plain H.v, CLT) or from a counter (CR Lanczos) --
// so the whole grid works on one contiguous window of rows at a time.

}  // namespace ftlm
