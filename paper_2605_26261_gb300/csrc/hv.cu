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

template <typename V> __device__ __forceinline__ V jh_of(const BondTable &bt, int b);
template <> __device__ __forceinline__ float jh_of<float>(const BondTable &bt, int b) { return bt.jhf[b]; }
template <> __device__ __forceinline__ double jh_of<double>(const BondTable &bt, int b) { return bt.jh[b]; }
template <typename V> __device__ __forceinline__ V jsum4_of(const BondTable &bt);
template <> __device__ __forceinline__ float jsum4_of<float>(const BondTable &bt) { return bt.jsum4f; }
template <> __device__ __forceinline__ double jsum4_of<double>(const BondTable &bt) { return bt.jsum4; }

struct EpiDev {
    ChainState *st;
    double *partials;
    double *alpha_out;
    int has_prev;
};

template <typename V, bool CLT, bool LANCZOS>
__global__ void __launch_bounds__(kRowThreads)
hv_kernel(const SectorTables s, const BondTable bt, const V *__restrict__ x, V *y, const EpiDev ep)
{
    extern __shared__ uint16_t s_tlo[];
    double inv_s = 1.0, c_prev = 0.0;
    if (LANCZOS) {
        const ChainState *st = ep.st;
        if (st->stopped) return;  // chain ended: grid-uniform
        inv_s = 1.0 / st->s_cur;
        if (ep.has_prev) c_prev = st->beta_prev / st->s_prev;
    }
    if (!CLT) {
        for (uint32_t i = threadIdx.x; i <= s.lomask; i += blockDim.x) s_tlo[i] = __ldg(s.tlo + i);
        __syncthreads();
    }
    const V inv_s_v = (V)inv_s, c_prev_v = (V)c_prev, jsum4 = jsum4_of<V>(bt);
    double apart = 0.0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < s.D; t += stride) {
        V acc = 0, dsum = 0;
        if (CLT) {
            const uint32_t n = __ldcs(s.basis + t);
#pragma unroll 4
            for (int b = 0; b < bt.nb; ++b) {
                const uint32_t m = bt.mlo[b], xm = n & m;
                if (xm != 0u && xm != m) {
                    const uint32_t nn = n ^ m;
                    const uint2 e = __ldg(s.clt + (nn >> 5));
                    const uint32_t k = e.y + __popc(e.x & ((1u << (nn & 31u)) - 1u));
                    const V jh = jh_of<V>(bt, b);
                    acc = fma(jh, __ldg(x + k), acc);
                    dsum += jh;
                }
            }
        } else {
            // inverse map t -> (h, l)
            uint32_t lo = 0, hi = s.H;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (__ldg(s.thi + mid) <= t) lo = mid;
                else hi = mid;
            }
            const uint32_t h = lo, r_hi = __ldg(s.thi + h), r_lo = t - r_hi;
            const uint32_t l = __ldg(s.ulo + __ldg(s.uoff + (s.K - __popc(h))) + r_lo);
            const int b1 = bt.n_lo, b2 = bt.n_lo + bt.n_hi;
#pragma unroll 4
            for (int b = 0; b < b1; ++b) {  // both sites in the low block
                const uint32_t m = bt.mlo[b], xm = l & m;
                if (xm != 0u && xm != m) {
                    const uint32_t k = r_hi + s_tlo[l ^ m];
                    const V jh = jh_of<V>(bt, b);
                    acc = fma(jh, __ldg(x + k), acc);
                    dsum += jh;
                }
            }
#pragma unroll 4
            for (int b = b1; b < b2; ++b) {  // both sites in the high block
                const uint32_t m = bt.mhi[b], xm = h & m;
                if (xm != 0u && xm != m) {
                    const uint32_t k = __ldg(s.thi + (h ^ m)) + r_lo;
                    const V jh = jh_of<V>(bt, b);
                    acc = fma(jh, __ldg(x + k), acc);
                    dsum += jh;
                }
            }
#pragma unroll 4
            for (int b = b2; b < bt.nb; ++b) {  // one site in each block
                const uint32_t ml = bt.mlo[b], mh = bt.mhi[b];
                if (((l & ml) != 0u) != ((h & mh) != 0u)) {
                    const uint32_t k = __ldg(s.thi + (h ^ mh)) + s_tlo[l ^ ml];
                    const V jh = jh_of<V>(bt, b);
                    acc = fma(jh, __ldg(x + k), acc);
                    dsum += jh;
                }
            }
        }
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

template <typename V, bool CLT, bool LANCZOS>
ftlm_status launch(const ftlm_basis *b, const V *x, V *y, const EpiDev &ep, cudaStream_t stream)
{
    static int occ = -1;  // resident blocks per SM for this instantiation
    const size_t smem = CLT ? 0 : ((size_t)1 << b->L) * sizeof(uint16_t);
    auto kern = hv_kernel<V, CLT, LANCZOS>;
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

template <typename V>
ftlm_status launch_typed(const ftlm_basis *b, const void *x, void *y, const LanczosHv *epi,
                         cudaStream_t stream)
{
    EpiDev ep{};
    const bool clt = b->mode == FTLM_RANK_CLT;
    if (epi) {
        ep.st = epi->st;
        ep.partials = epi->partials;
        ep.alpha_out = epi->alpha_out;
        ep.has_prev = epi->j > 1;
        return clt ? launch<V, true, true>(b, (const V *)x, (V *)y, ep, stream)
                   : launch<V, false, true>(b, (const V *)x, (V *)y, ep, stream);
    }
    return clt ? launch<V, true, false>(b, (const V *)x, (V *)y, ep, stream)
               : launch<V, false, false>(b, (const V *)x, (V *)y, ep, stream);
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
