// Row work of the general-spin H.v (Eq. 12-14 for any s), shared by the
// single-sector kernel (spin.cu) and the multi-sector path (msv.cu): the inverse
// map of a row to its base-d digits, the digit-block rank of a source label, and
// the per-row sums of the two ladder terms of every bond (gathers of a chunk of
// bonds issued together, predicated).
#pragma once

#include "ftlm_internal.cuh"
#include "vec.cuh"

namespace ftlm {

constexpr int kSpinMaxSites = 16;           // 4-bit digit fields in 64 bits
constexpr int kSpinMaxTwoS = 7;             // d <= 8
constexpr uint64_t kSpinMaxLow = 1u << 14;  // tlo entries (shared memory)
constexpr uint64_t kSpinMaxHigh = 1u << 27; // thi entries

__device__ __forceinline__ uint32_t div_d(const SpinDev &p, uint32_t n)
{
    return (uint32_t)(((uint64_t)n * p.magic) >> p.shift);
}

// thi[h]: from a shared-memory copy (TS) or through the read-only global path.
template <bool TS> __device__ __forceinline__ uint32_t thi_at(const SectorTables &s, const uint32_t *s_thi, uint32_t h)
{
    if constexpr (TS) return s_thi[h];
    else return __ldg(s.thi + h);
}

struct SpinRow {
    uint32_t lo, hi;      // low and high labels of the row
    uint32_t thi_h, r_lo; // the row's two halves of its rank
    uint64_t dig;         // digit k in bits 4k .. 4k+3
};

template <bool TS>
__device__ __forceinline__ void spin_unrank(const SectorTables &s, const SpinDev &p, const uint32_t *s_thi, uint32_t t,
                                            SpinRow &w)
{
    const uint32_t kc = t >> kHsShift;
    uint32_t lo = __ldg(s.hs + kc), hi = __ldg(s.hs + kc + 1) + 1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (thi_at<TS>(s, s_thi, mid) <= t) lo = mid;
        else hi = mid;
    }
    w.hi = lo;
    w.thi_h = thi_at<TS>(s, s_thi, lo);
    w.r_lo = t - w.thi_h;
    uint64_t dig = 0;
    uint32_t n = w.hi, sum = 0;
    for (int k = s.L; k < s.N; ++k) {
        const uint32_t q = div_d(p, n), a = n - q * p.d;
        dig |= (uint64_t)a << (4 * k);
        sum += a;
        n = q;
    }
    w.lo = __ldg(s.ulo + __ldg(s.uoff + (p.A - sum)) + w.r_lo);
    n = w.lo;
    for (int k = 0; k < s.L; ++k) {
        const uint32_t q = div_d(p, n), a = n - q * p.d;
        dig |= (uint64_t)a << (4 * k);
        n = q;
    }
    w.dig = dig;
}

// Rank of the row's label with digit i moved by di and digit j by dj (+-1).
template <bool TS>
__device__ __forceinline__ uint32_t spin_rank(const SectorTables &s, const uint16_t *s_tlo, const uint32_t *s_thi,
                                              const SpinRow &w, uint32_t flags, uint32_t pi, uint32_t pj, int di)
{
    uint32_t lo = w.lo, hi = w.hi;
    const uint32_t ai = di > 0 ? pi : 0u - pi, aj = di > 0 ? 0u - pj : pj;
    if (flags & 1u) hi += ai;
    else lo += ai;
    if (flags & 2u) hi += aj;
    else lo += aj;
    // a valid move keeps both labels in range; the clamps only bound the addresses
    // of a move that the caller discards
    lo = min(lo, s.lomask);
    hi = min(hi, s.H - 1u);
    const uint32_t rh = hi == w.hi ? w.thi_h : thi_at<TS>(s, s_thi, hi);
    const uint32_t rl = lo == w.lo ? w.r_lo : (uint32_t)s_tlo[lo];
    return rh + rl;
}

template <typename V> __device__ __forceinline__ const V *spin_J(const SpinDev &p);
template <> __device__ __forceinline__ const float *spin_J<float>(const SpinDev &p) { return p.jf; }
template <> __device__ __forceinline__ const double *spin_J<double>(const SpinDev &p) { return p.jd; }
template <typename V> __device__ __forceinline__ const V *spin_up(const SpinDev &p);
template <> __device__ __forceinline__ const float *spin_up<float>(const SpinDev &p) { return p.upf; }
template <> __device__ __forceinline__ const double *spin_up<double>(const SpinDev &p) { return p.upd; }

// Per-bond factors of a row, indexed by the digit pair d a_i + a_j (d <= 8):
// [0, 64) the s_i^+ s_j^- factor of Eq. 13 and [64, 128) the s_i^- s_j^+ factor of
// Eq. 14, both with the 1/2 of Eq. 12 and zero where the source digit leaves
// 0 .. 2s; [128, 192) m_i m_j (exact: products of half-integers).  The compact
// index keeps the d^2 entries of a table in distinct shared-memory banks for
// d <= 5, so the lanes of a warp read them without bank conflicts.
constexpr int kSpinCoef = 3 * 64;

template <typename V> __device__ __forceinline__ void spin_stage_coef(const SpinDev &p, V *s_cf)
{
    const V *up = spin_up<V>(p);
    const uint32_t two_s = p.two_s, d = p.d;
    const V sv = (V)(0.5 * p.two_s);
    for (uint32_t idx = threadIdx.x; idx < (uint32_t)kSpinCoef; idx += blockDim.x) {
        const uint32_t tab = idx >> 6, rem = idx & 63u, ai = rem / d, aj = rem % d;
        V v = (V)0;
        if (rem < d * d) {
            if (tab == 0u && ai >= 1u && aj < two_s) v = (V)0.5 * up[ai - 1] * up[aj];
            else if (tab == 1u && ai < two_s && aj >= 1u) v = (V)0.5 * up[ai] * up[aj - 1];
            else if (tab == 2u) v = ((V)ai - sv) * ((V)aj - sv);
        }
        s_cf[idx] = v;
    }
}

// Bonds per chunk (two gathers each); build option FTLM_SPIN_CHUNK_B8 for B = 8.
#ifndef FTLM_SPIN_CHUNK_B8
#define FTLM_SPIN_CHUNK_B8 3
#endif
template <int B> __host__ __device__ constexpr int spin_chunk()
{
    return B >= 16 ? 1 : (B >= 8 ? FTLM_SPIN_CHUNK_B8 : 4);
}

// Row t: acc[r] = sum of the ladder terms of vector r, diag = sum_b J_b m_i m_j.
// TS: thi is staged in shared memory at s_thi (else s_thi is unused).
template <typename V, int B, int C, bool TS>
__device__ __forceinline__ void spin_row(const SectorTables &s, const SpinDev &p, const uint16_t *s_tlo,
                                         const uint32_t *s_thi, const uint4 *s_bond, const V *s_J, const V *s_cf,
                                         const V *__restrict__ x, uint32_t t, V (&acc)[B], V &diag)
{
    SpinRow w;
    spin_unrank<TS>(s, p, s_thi, t, w);
    diag = (V)0;
#pragma unroll
    for (int r = 0; r < B; ++r) acc[r] = (V)0;
    for (uint32_t b0 = 0; b0 < p.nb; b0 += C) {
        uint32_t k[2 * C];
        bool use[2 * C];
        V c[2 * C];
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const uint32_t b = b0 + q;
            const bool in = b < p.nb;
            const uint4 e = s_bond[in ? b : 0];
            const uint32_t i = e.x & 255u, j = (e.x >> 8) & 255u, flags = e.x >> 16;
            const uint32_t ai = (uint32_t)(w.dig >> (4 * i)) & 15u, aj = (uint32_t)(w.dig >> (4 * j)) & 15u;
            const uint32_t ij = ai * p.d + aj;
            const V J = in ? s_J[b] : (V)0;
            diag = fma(J, s_cf[128 + ij], diag);
            // a term exists where its factor is nonzero; the clamps of spin_rank keep
            // the table addresses of a dropped term in range
            const V f0 = s_cf[ij], f1 = s_cf[64 + ij];
            // s_i^+ s_j^-: source digits (a_i - 1, a_j + 1), coefficient Eq. 13
            use[2 * q] = in && f0 != (V)0;
            c[2 * q] = J * f0;
            k[2 * q] = use[2 * q] ? spin_rank<TS>(s, s_tlo, s_thi, w, flags, e.y, e.z, -1) : 0u;
            // s_i^- s_j^+: source digits (a_i + 1, a_j - 1), coefficient Eq. 14
            use[2 * q + 1] = in && f1 != (V)0;
            c[2 * q + 1] = J * f1;
            k[2 * q + 1] = use[2 * q + 1] ? spin_rank<TS>(s, s_tlo, s_thi, w, flags, e.y, e.z, +1) : 0u;
        }
        V xv[2 * C][B];
#pragma unroll
        for (int q = 0; q < 2 * C; ++q) {
            if (use[q]) {
                ld_vec<B>(x + (size_t)k[q] * B, xv[q], false);
            } else {
#pragma unroll
                for (int r = 0; r < B; ++r) xv[q][r] = (V)0;
            }
        }
#pragma unroll
        for (int q = 0; q < 2 * C; ++q)
#pragma unroll
            for (int r = 0; r < B; ++r) acc[r] = fma(c[q], xv[q][r], acc[r]);
    }
}

}  // namespace ftlm
