// Row work of the general-spin H.v (Eq. 12-14 for any s), shared by the
// single-sector kernel (spin.cu) and the multi-sector path (msv.cu): the inverse
// map of a row to its base-d digits, and the per-row sums of the two ladder terms
// of every bond, class by class (both sites in the low digit block, both in the
// high block, one in each), each class with its own digit-block rank arithmetic
// (gathers of a chunk of bonds issued together, predicated).
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

// The bonds [b_beg, b_end) of one class of row w: the two ladder terms of each,
// with the rank arithmetic of the class (CLS 0: both sites in the low block, only
// the low half of the rank moves; 1: both in the high block; 2: site i low, site j
// high).  Adds J m_i m_j to diag and the terms to acc.  A term whose factor is zero
// does not exist; the clamps keep the table addresses of such a term in range.
template <typename V, int B, int C, bool TS, int CLS>
__device__ __forceinline__ void spin_class(const SectorTables &s, const SpinDev &p, const uint16_t *s_tlo,
                                           const uint32_t *s_thi, const uint4 *s_bond, const V *s_J, const V *s_cf,
                                           const V *__restrict__ x, const SpinRow &w, uint32_t b_beg, uint32_t b_end,
                                           V (&acc)[B], V &diag)
{
    for (uint32_t b0 = b_beg; b0 < b_end; b0 += C) {
        uint32_t k[2 * C];
        bool use[2 * C];
        V c[2 * C];
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const uint32_t b = b0 + q;
            const bool in = b < b_end;
            const uint4 e = s_bond[in ? b : b_beg];
            const uint32_t i = e.x & 255u, j = (e.x >> 8) & 255u, pi = e.y, pj = e.z;
            const uint32_t ai = (uint32_t)(w.dig >> (4 * i)) & 15u, aj = (uint32_t)(w.dig >> (4 * j)) & 15u;
            const uint32_t ij = ai * p.d + aj;
            const V J = in ? s_J[b] : (V)0;
            diag = fma(J, s_cf[128 + ij], diag);
            const V f0 = s_cf[ij], f1 = s_cf[64 + ij];
            use[2 * q] = in && f0 != (V)0;      // s_i^+ s_j^-: source digits (a_i - 1, a_j + 1), Eq. 13
            use[2 * q + 1] = in && f1 != (V)0;  // s_i^- s_j^+: source digits (a_i + 1, a_j - 1), Eq. 14
            c[2 * q] = J * f0;
            c[2 * q + 1] = J * f1;
            uint32_t k0, k1;
            if constexpr (CLS == 0) {
                k0 = w.thi_h + s_tlo[min(w.lo - pi + pj, s.lomask)];
                k1 = w.thi_h + s_tlo[min(w.lo + pi - pj, s.lomask)];
            } else if constexpr (CLS == 1) {
                k0 = thi_at<TS>(s, s_thi, min(w.hi - pi + pj, s.H - 1u)) + w.r_lo;
                k1 = thi_at<TS>(s, s_thi, min(w.hi + pi - pj, s.H - 1u)) + w.r_lo;
            } else {
                k0 = thi_at<TS>(s, s_thi, min(w.hi + pj, s.H - 1u)) + s_tlo[min(w.lo - pi, s.lomask)];
                k1 = thi_at<TS>(s, s_thi, min(w.hi - pj, s.H - 1u)) + s_tlo[min(w.lo + pi, s.lomask)];
            }
            k[2 * q] = use[2 * q] ? k0 : 0u;
            k[2 * q + 1] = use[2 * q + 1] ? k1 : 0u;
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
    const uint32_t e_ll = p.n_ll, e_hh = p.n_ll + p.n_hh;
    spin_class<V, B, C, TS, 0>(s, p, s_tlo, s_thi, s_bond, s_J, s_cf, x, w, 0u, e_ll, acc, diag);
    spin_class<V, B, C, TS, 1>(s, p, s_tlo, s_thi, s_bond, s_J, s_cf, x, w, e_ll, e_hh, acc, diag);
    spin_class<V, B, C, TS, 2>(s, p, s_tlo, s_thi, s_bond, s_J, s_cf, x, w, e_hh, p.nb, acc, diag);
}

}  // namespace ftlm
