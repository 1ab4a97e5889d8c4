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
// Lanczos epilogue (Paige's ordering).  The stored vector u_j is un-normalized,
// q_j = u_j / s_j.  With x = u_j and the in-place buffer holding u_{j-1}:
//   y[t] = (H u_j)[t] / s_j - (beta_{j-1} / s_{j-1}) u_{j-1}[t]     (overwrites u_{j-1})
//   alpha partial += q_j[t] y[t]                                    (FP64)
// The last block adds the per-block partials in a fixed order and stores alpha_j.
#include "ftlm_internal.cuh"
#include "reduce.cuh"

namespace ftlm {

namespace {

struct EpiDev {
    ChainState *st;
    double *partials;
    double *alpha_out;
    int has_prev;
};

// J/2 of a bond slot in the vector type.
template <typename V> __device__ __forceinline__ V slot_jh(const uint4 &e);
template <> __device__ __forceinline__ float slot_jh<float>(const uint4 &e) { return __uint_as_float(e.z); }
template <> __device__ __forceinline__ double slot_jh<double>(const uint4 &e)
{
    return __hiloint2double((int)e.w, (int)e.z);
}

template <typename Lbl>
__device__ __forceinline__ Lbl slot_mask(const uint4 &e)
{
    if constexpr (sizeof(Lbl) == 8) return (Lbl)e.x | ((Lbl)e.y << 32);
    else return e.x;
}

// Gather the chunk's antiparallel terms (predicated loads, all issued together).
template <typename V>
__device__ __forceinline__ void gather_accumulate(const V *__restrict__ x, const bool (&aa)[kBondChunk],
                                                  const uint32_t (&kk)[kBondChunk],
                                                  const V (&jh)[kBondChunk], V &acc, V &dsum)
{
    V xv[kBondChunk];
#pragma unroll
    for (int q = 0; q < kBondChunk; ++q) xv[q] = aa[q] ? __ldg(x + kk[q]) : (V)0;
#pragma unroll
    for (int q = 0; q < kBondChunk; ++q) {
        acc = fma(jh[q], xv[q], acc);
        if (aa[q]) dsum += jh[q];
    }
}

// Row sums of one output row (CR): sum over antiparallel bonds of (J_b/2) x[k_b]
// in acc, sum of their J_b/2 in dsum.
template <typename V, typename Lbl>
__device__ __forceinline__ void row_cr(const SectorTables &s, const BondList &bl, const uint4 *s_bond,
                                       const uint16_t *s_tlo, const V *__restrict__ x, uint32_t t, V &acc,
                                       V &dsum)
{
    // inverse map t -> (h, l): last h with thi[h] <= t, then ulo within its group
    uint32_t lo = 0, hi = s.H;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(s.thi + mid) <= t) lo = mid;
        else hi = mid;
    }
    const uint32_t h = lo, r_hi = __ldg(s.thi + h), r_lo = t - r_hi;
    const uint32_t l = __ldg(s.ulo + __ldg(s.uoff + (s.K - __popc(h))) + r_lo);
    bool aa[kBondChunk];
    uint32_t kk[kBondChunk];
    V jh[kBondChunk];
    const int e_lo = bl.n_lo, e_hi = bl.n_lo + bl.n_hi;
    for (int b0 = 0; b0 < e_lo; b0 += kBondChunk) {  // both sites in the low block
#pragma unroll
        for (int q = 0; q < kBondChunk; ++q) {
            const uint4 e = s_bond[b0 + q];
            const uint32_t m = e.x, xm = l & m;
            aa[q] = (xm != 0u) & (xm != m);
            kk[q] = r_hi + s_tlo[l ^ m];
            jh[q] = slot_jh<V>(e);
        }
        gather_accumulate(x, aa, kk, jh, acc, dsum);
    }
    for (int b0 = e_lo; b0 < e_hi; b0 += kBondChunk) {  // both sites in the high block
#pragma unroll
        for (int q = 0; q < kBondChunk; ++q) {
            const uint4 e = s_bond[b0 + q];
            const uint32_t m = e.y, xm = h & m;
            aa[q] = (xm != 0u) & (xm != m);
            kk[q] = __ldg(s.thi + (h ^ m)) + r_lo;
            jh[q] = slot_jh<V>(e);
        }
        gather_accumulate(x, aa, kk, jh, acc, dsum);
    }
    const Lbl n = ((Lbl)h << s.L) | l;
    for (int b0 = e_hi; b0 < bl.nb; b0 += kBondChunk) {  // any bond
#pragma unroll
        for (int q = 0; q < kBondChunk; ++q) {
            const uint4 e = s_bond[b0 + q];
            const Lbl m = slot_mask<Lbl>(e), xm = n & m, nn = n ^ m;
            aa[q] = (xm != 0) & (xm != m);
            kk[q] = __ldg(s.thi + (uint32_t)(nn >> s.L)) + s_tlo[(uint32_t)nn & s.lomask];
            jh[q] = slot_jh<V>(e);
        }
        gather_accumulate(x, aa, kk, jh, acc, dsum);
    }
}

// Row sums of one output row (CLT, Algorithm 2 per exchanged label).
template <typename V>
__device__ __forceinline__ void row_clt(const SectorTables &s, const BondList &bl, const uint4 *s_bond,
                                        const V *__restrict__ x, uint32_t t, V &acc, V &dsum)
{
    const uint32_t n = __ldcs(s.basis + t);
    bool aa[kBondChunk];
    uint32_t kk[kBondChunk], nn[kBondChunk];
    uint2 e2[kBondChunk];
    V jh[kBondChunk];
    for (int b0 = 0; b0 < bl.nb; b0 += kBondChunk) {
#pragma unroll
        for (int q = 0; q < kBondChunk; ++q) {
            const uint4 e = s_bond[b0 + q];
            const uint32_t m = e.x, xm = n & m;
            aa[q] = (xm != 0u) & (xm != m);
            nn[q] = n ^ m;
            jh[q] = slot_jh<V>(e);
        }
#pragma unroll
        for (int q = 0; q < kBondChunk; ++q) e2[q] = aa[q] ? __ldg(s.clt + (nn[q] >> 5)) : make_uint2(0u, 0u);
#pragma unroll
        for (int q = 0; q < kBondChunk; ++q) kk[q] = e2[q].y + __popc(e2[q].x & ((1u << (nn[q] & 31u)) - 1u));
        gather_accumulate(x, aa, kk, jh, acc, dsum);
    }
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS>
__global__ void __launch_bounds__(kRowThreads)
hv_kernel(const SectorTables s, const BondList bl, const V *__restrict__ x, V *y, const EpiDev ep)
{
    extern __shared__ uint16_t s_tlo[];
    __shared__ uint4 s_bond[kMaxBondSlots];
    double inv_s = 1.0, c_prev = 0.0;
    if (LANCZOS) {
        const ChainState *st = ep.st;
        if (st->stopped) return;  // chain ended: grid-uniform
        inv_s = 1.0 / st->s_cur;
        if (ep.has_prev) c_prev = st->beta_prev / st->s_prev;
    }
    {
        const uint4 *src = sizeof(V) == 4 ? bl.slots_f32 : bl.slots_f64;
        for (int i = threadIdx.x; i < bl.nb; i += blockDim.x) s_bond[i] = src[i];
    }
    if (!CLT)
        for (uint32_t i = threadIdx.x; i <= s.lomask; i += blockDim.x) s_tlo[i] = __ldg(s.tlo + i);
    __syncthreads();
    const V inv_s_v = (V)inv_s, c_prev_v = (V)c_prev, jsum4 = (V)bl.jsum4;
    double apart = 0.0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < s.D; t += stride) {
        V acc = 0, dsum = 0;
        if (CLT) row_clt<V>(s, bl, s_bond, x, t, acc, dsum);
        else row_cr<V, Lbl>(s, bl, s_bond, s_tlo, x, t, acc, dsum);
        const V xt = __ldg(x + t);
        const V hv = fma(jsum4 - dsum, xt, acc);
        if (LANCZOS) {
            const V up = ep.has_prev ? __ldcs(y + t) : (V)0;
            const V yv = fma(-c_prev_v, up, hv * inv_s_v);
            __stcs(y + t, yv);
            apart += (double)(xt * inv_s_v) * (double)yv;
        } else {
            __stcs(y + t, hv);
        }
    }
    if (LANCZOS) {
        const double part = block_sum<kRowThreads>(apart);
        if (publish_partial(part, ep.partials, &ep.st->counter) && threadIdx.x < 32) {
            const double alpha = total_of_partials(ep.partials, gridDim.x);
            if (threadIdx.x == 0) {
                ep.st->alpha = alpha;
                *ep.alpha_out = alpha;
                ep.st->counter = 0;
            }
        }
    }
}

template <typename V, typename Lbl, bool CLT, bool LANCZOS>
ftlm_status launch(const ftlm_basis *b, const V *x, V *y, const EpiDev &ep, cudaStream_t stream)
{
    static int occ = -1;  // resident blocks per SM for this instantiation
    const size_t smem = CLT ? 0 : ((size_t)1 << b->L) * sizeof(uint16_t);
    auto kern = hv_kernel<V, Lbl, CLT, LANCZOS>;
    if (occ < 0) {
        const size_t smem_max = CLT ? 0 : ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
        FTLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRowThreads, smem_max));
    }
    const int grid = row_grid(b, b->D, occ);
    void *tok = profile_begin(kProfHv, stream);
    kern<<<grid, kRowThreads, smem, stream>>>(b->tables(), CLT ? b->bonds_clt : b->bonds_cr, x, y, ep);
    profile_end(tok, stream);
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V, bool LANCZOS>
ftlm_status launch_mode(const ftlm_basis *b, const void *x, void *y, const EpiDev &ep, cudaStream_t stream)
{
    if (b->mode == FTLM_RANK_CLT) return launch<V, uint32_t, true, LANCZOS>(b, (const V *)x, (V *)y, ep, stream);
    if (b->N <= 32) return launch<V, uint32_t, false, LANCZOS>(b, (const V *)x, (V *)y, ep, stream);
    return launch<V, uint64_t, false, LANCZOS>(b, (const V *)x, (V *)y, ep, stream);
}

template <typename V>
ftlm_status launch_typed(const ftlm_basis *b, const void *x, void *y, const LanczosHv *epi,
                         cudaStream_t stream)
{
    EpiDev ep{};
    if (epi) {
        ep.st = epi->st;
        ep.partials = epi->partials;
        ep.alpha_out = epi->alpha_out;
        ep.has_prev = epi->j > 1;
        return launch_mode<V, true>(b, x, y, ep, stream);
    }
    return launch_mode<V, false>(b, x, y, ep, stream);
}

}  // namespace

ftlm_status launch_hv(const ftlm_basis *b, ftlm_dtype dtype, const void *x, void *y,
                      const LanczosHv *epi, cudaStream_t stream)
{
    return dtype == FTLM_F32 ? launch_typed<float>(b, x, y, epi, stream)
                             : launch_typed<double>(b, x, y, epi, stream);
}

}  // namespace ftlm

extern "C" ftlm_status ftlm_hv(const ftlm_basis *b, ftlm_dtype dtype, const void *x_dev, void *y_dev,
                               void *stream)
{
    if (!b) return ftlm::fail(FTLM_EINVAL, "NULL basis");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return ftlm::fail(FTLM_EINVAL, "bad dtype");
    if (!x_dev || !y_dev) return ftlm::fail(FTLM_EINVAL, "NULL vector");
    if (x_dev == y_dev) return ftlm::fail(FTLM_EINVAL, "x and y must not overlap");
    if (((uintptr_t)x_dev | (uintptr_t)y_dev) & 15u) return ftlm::fail(FTLM_EINVAL, "vectors must be 16-byte aligned");
    return ftlm::launch_hv(b, dtype, x_dev, y_dev, nullptr, (cudaStream_t)stream);
}
