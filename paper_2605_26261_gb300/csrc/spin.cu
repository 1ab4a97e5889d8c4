// General local spin s >= 1 (two_s = 2s >= 2): sector setup, labels/ranks and the
// H.v gather with its Lanczos epilogue (Sec. 2: Eq. 11-17 with d = 2s + 1).
//
// Labels.  A state is the label n = sum_k a_k d^k (Eq. 11), a_k = m_k + s the k-th
// base-d digit; the sector of total S^z = M holds the labels with digit sum
// A = N s + M (Eq. 17), numbered in increasing label order.
//
// Rank.  Algorithm 1 adds, at every digit position p from the top, the number of
// sector labels whose digits above p agree and whose digit p is smaller:
// D_c(p, A_p, a_p) of Eq. 16 with A_p the digit sum still to place.  As for spin
// 1/2, the L low positions and the N - L high positions are each collapsed into one
// table lookup: the low positions contribute tlo[n_lo] (n_lo = n mod d^L; within a
// sector their remaining sum is the digit sum of n_lo itself) and the high
// positions contribute thi[n_hi] (n_hi = n div d^L), which is also the number of
// sector labels below n_hi d^L.  So rank(n) = thi[n_hi] + tlo[n_lo], bit-identical
// to Algorithm 1.  d^L <= 2^14 keeps tlo in shared memory (16-bit entries).
//
// Row.  The inverse map of row t binary-searches thi (bounded by the coarse row
// index), takes the low label from ulo (low labels grouped by digit sum), and
// unpacks all N digits into 4-bit fields.  Per bond the two ladder terms of Eq. 12
// have the coefficients of Eq. 13 and Eq. 14; a term exists when the source digits
// stay in 0 .. 2s.  A move changes the labels by +-d^i and -+d^j; a bond with both
// sites in one block keeps the other block's half of the rank.  Gathers of a chunk
// of bonds are issued together (predicated), then accumulated.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "epi.cuh"
#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "spin_rows.cuh"
#include "vec.cuh"

namespace ftlm {

namespace {


uint64_t ipow(uint64_t d, int k)
{
    uint64_t p = 1;
    for (int i = 0; i < k; ++i) p *= d;
    return p;
}

// D(m, a) of Eq. 15 (digit strings of length m, digits 0..two_s, sum a), m <= N.
struct Dims {
    int two_s, amax;
    std::vector<uint64_t> v;  // (N + 1) x (amax + 1)
    Dims(int N, int two_s_) : two_s(two_s_), amax(N * two_s_), v((size_t)(N + 1) * (N * two_s_ + 1), 0)
    {
        v[0] = 1;
        for (int m = 1; m <= N; ++m)
            for (int a = 0; a <= amax; ++a) {
                uint64_t c = 0;
                for (int q = 0; q <= two_s && q <= a; ++q) c += at(m - 1, a - q);
                v[(size_t)m * (amax + 1) + a] = c;
            }
    }
    uint64_t at(int m, int a) const { return (a < 0 || a > amax) ? 0 : v[(size_t)m * (amax + 1) + a]; }
};

// Resident CTAs per SM the registers are capped for; build option
// FTLM_SPIN_B8_MIN_CTAS for B >= 8 (FP64 blocks of 4: 2, other blocks: 3).
#ifndef FTLM_SPIN_B8_MIN_CTAS
#define FTLM_SPIN_B8_MIN_CTAS 2
#endif

// High-block rank tables up to this many entries (64 KB) are staged in shared
// memory next to tlo, taking the lookup of the high half of a source rank off the
// global load path; build option FTLM_SPIN_SMEM_HIGH (0: never).
#ifndef FTLM_SPIN_SMEM_HIGH
#define FTLM_SPIN_SMEM_HIGH 16384
#endif
constexpr uint64_t kSpinSmemHigh = FTLM_SPIN_SMEM_HIGH;

template <typename V, bool LANCZOS, int B, bool TS>
__global__ void __launch_bounds__(kRowThreads, B >= 8 ? FTLM_SPIN_B8_MIN_CTAS : (sizeof(V) == 8 && B >= 4 ? 2 : 3))
hv_spin_kernel(const SectorTables s, const SpinDev p, const V *__restrict__ x, V *y, const EpiDev ep)
{
    constexpr int C = spin_chunk<B>();
    extern __shared__ uint16_t s_tlo[];
    // thi after tlo, at a 16-byte boundary (tlo has at most 2^14 entries)
    uint32_t *s_thi = reinterpret_cast<uint32_t *>(s_tlo + (((size_t)s.lomask + 8) & ~(size_t)7));
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ V s_J[kMaxBondSlots];
    __shared__ V s_cf[kSpinCoef];
    __shared__ V s_inv_s[B], s_c_prev[B];
    if (LANCZOS && epi_begin<V, B>(ep, s_inv_s, s_c_prev)) return;
    for (uint32_t i = threadIdx.x; i < p.nb; i += blockDim.x) {
        s_bond[i] = p.slots[i];
        s_J[i] = spin_J<V>(p)[i];
    }
    spin_stage_coef<V>(p, s_cf);
    for (uint32_t i = threadIdx.x; i <= s.lomask; i += blockDim.x) s_tlo[i] = __ldg(s.tlo + i);
    if (TS)
        for (uint32_t i = threadIdx.x; i < s.H; i += blockDim.x) s_thi[i] = __ldg(s.thi + i);
    __syncthreads();

    DotAcc<V> apart[B];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ntiles = (uint32_t)(((uint64_t)s.D + 31u) / 32u);
    for (uint32_t tile = warp; tile < ntiles; tile += nwarps) {
        const uint32_t tt = tile * 32u + lane;
        const bool ok_row = tt < s.D;
        const uint32_t t = ok_row ? tt : s.D - 1;  // rows past the end recompute the last row, unstored
        V acc[B], diag;
        spin_row<V, B, C, TS>(s, p, s_tlo, s_thi, s_bond, s_J, s_cf, x, t, acc, diag);
        if (ok_row) epi_row<V, B, LANCZOS>(ep, s_inv_s, s_c_prev, x, y, t, diag, acc, apart);
    }
    if (LANCZOS) epi_end<V, B, kRowThreads>(ep, apart);
}

__global__ void spin_labels_kernel(SectorTables s, SpinDev p, uint64_t low_size, uint64_t first, uint64_t count,
                                   uint64_t *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        SpinRow w;
        spin_unrank<false>(s, p, nullptr, (uint32_t)(first + i), w);
        out[i] = (uint64_t)w.hi * low_size + w.lo;
    }
}

// Rank of arbitrary labels; -1 outside the sector (a digit sum other than A, or a
// label >= d^N).
__global__ void spin_rank_kernel(SectorTables s, SpinDev p, uint64_t low_size, uint64_t high_size, uint64_t count,
                                 const uint64_t *labels, int64_t *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t n = labels[i];
        const uint64_t hi = n / low_size, lo = n - hi * low_size;
        int64_t r = -1;
        if (hi < high_size) {
            uint32_t sum = 0;
            uint64_t m = n;
            for (int k = 0; k < s.N; ++k) {
                sum += (uint32_t)(m % p.d);
                m /= p.d;
            }
            if (sum == p.A) r = (int64_t)__ldg(s.thi + hi) + __ldg(s.tlo + lo);
        }
        out[i] = r;
    }
}

int grid_of(const ftlm_basis *b, uint64_t n)
{
    const uint64_t g = (n + 255) / 256, cap = (uint64_t)b->num_sms * 16;
    return (int)std::max<uint64_t>(1, std::min(g, cap));
}

template <typename V, bool LANCZOS, int B>
ftlm_status launch_spin(const ftlm_basis *b, const V *x, V *y, const EpiDev &ep, cudaStream_t stream)
{
    const bool ts = b->H <= kSpinSmemHigh;
    auto kern = ts ? hv_spin_kernel<V, LANCZOS, B, true> : hv_spin_kernel<V, LANCZOS, B, false>;
    const size_t tlo_bytes = (((size_t)b->tables().lomask + 8) & ~(size_t)7) * sizeof(uint16_t);
    const size_t smem_max = kSpinMaxLow * sizeof(uint16_t) + (ts ? kSpinSmemHigh * sizeof(uint32_t) : 0);
    int occ = 1;
    FTLM_CUDA(kernel_occupancy((const void *)kern, kRowThreads, smem_max, true, &occ));
    const size_t smem = tlo_bytes + (ts ? (size_t)b->H * sizeof(uint32_t) : 0);
    const int grid = row_grid(b, b->D, occ);
    void *tok = profile_begin(kProfHv, stream, B);
    kern<<<grid, kRowThreads, smem, stream>>>(b->tables(), b->spin, x, y, ep);
    note_launch();
    profile_end(tok, stream);
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V, bool LANCZOS>
ftlm_status launch_spin_b(const ftlm_basis *b, int B, const void *x, void *y, const EpiDev &ep,
                          cudaStream_t stream)
{
    const V *xv = (const V *)x;
    V *yv = (V *)y;
    switch (B) {
    case 4: return launch_spin<V, LANCZOS, 4>(b, xv, yv, ep, stream);
    case 8: return launch_spin<V, LANCZOS, 8>(b, xv, yv, ep, stream);
    case 16: return launch_spin<V, LANCZOS, 16>(b, xv, yv, ep, stream);
    default: return launch_spin<V, LANCZOS, 1>(b, xv, yv, ep, stream);
    }
}

}  // namespace

ftlm_status launch_hv_spin(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y,
                           const LanczosHv *epi, cudaStream_t stream)
{
    const EpiDev ep = epi_of(epi);
    if (dtype == FTLM_F32)
        return epi ? launch_spin_b<float, true>(b, B, x, y, ep, stream)
                   : launch_spin_b<float, false>(b, B, x, y, ep, stream);
    return epi ? launch_spin_b<double, true>(b, B, x, y, ep, stream)
               : launch_spin_b<double, false>(b, B, x, y, ep, stream);
}

ftlm_status launch_spin_labels(const ftlm_basis *b, uint64_t first, uint64_t count, uint64_t *out,
                               cudaStream_t stream)
{
    spin_labels_kernel<<<grid_of(b, count), 256, 0, stream>>>(b->tables(), b->spin, ipow(b->two_s + 1, b->L),
                                                              first, count, out);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

ftlm_status launch_spin_rank(const ftlm_basis *b, uint64_t count, const uint64_t *labels, int64_t *out,
                             cudaStream_t stream)
{
    spin_rank_kernel<<<grid_of(b, count), 256, 0, stream>>>(b->tables(), b->spin, ipow(b->two_s + 1, b->L),
                                                            b->H, count, labels, out);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_basis_create_spin(int N, int two_s, int two_sz, int n_bonds, const int *bi,
                                              const int *bj, const double *J, void *stream_, ftlm_basis **out)
{
    return basis_create_spin(N, two_s, two_sz, n_bonds, bi, bj, J, (cudaStream_t)stream_, true, out);
}

// wait: return once the tables are built (else once their build is queued).
ftlm_status ftlm::basis_create_spin(int N, int two_s, int two_sz, int n_bonds, const int *bi, const int *bj,
                                    const double *J, cudaStream_t stream_, bool wait, ftlm_basis **out)
{
    if (!out) return fail(FTLM_EINVAL, "out is NULL");
    *out = nullptr;
    if (two_s < 1) return fail(FTLM_EINVAL, "two_s < 1");
    if (two_s == 1) return basis_create_half(N, two_sz, n_bonds, bi, bj, J, FTLM_RANK_AUTO, stream_, wait, out);
    if (two_s > kSpinMaxTwoS) return fail(FTLM_EUNSUPPORTED, "spin above 7/2");
    if (N < 1) return fail(FTLM_EINVAL, "N out of range");
    if (N > kSpinMaxSites) return fail(FTLM_EUNSUPPORTED, "more than 16 sites at s > 1/2");
    if (two_sz < -N * two_s || two_sz > N * two_s || ((two_sz + N * two_s) & 1)) return fail(FTLM_EINVAL, "bad two_sz");
    if (n_bonds < 0) return fail(FTLM_EINVAL, "n_bonds < 0");
    if (n_bonds > FTLM_MAX_BONDS) return fail(FTLM_EUNSUPPORTED, "more than FTLM_MAX_BONDS bonds");
    if (n_bonds > 0 && (!bi || !bj || !J)) return fail(FTLM_EINVAL, "bond arrays are NULL");
    std::vector<std::pair<int, int>> seen;
    for (int k = 0; k < n_bonds; ++k) {
        const int i = std::min(bi[k], bj[k]), j = std::max(bi[k], bj[k]);
        if (i < 0 || j >= N) return fail(FTLM_EINVAL, "bond site out of range");
        if (i == j) return fail(FTLM_EINVAL, "bond joins a site to itself");
        if (!(J[k] == J[k]) || J[k] - J[k] != 0.0) return fail(FTLM_EINVAL, "non-finite coupling");
        seen.emplace_back(i, j);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return fail(FTLM_EINVAL, "duplicate bond");

    const int d = two_s + 1;
    const int A = (N * two_s + two_sz) / 2;
    const Dims dims(N, two_s);
    const uint64_t D = dims.at(N, A);
    if (D >= (1ull << 32)) return fail(FTLM_EUNSUPPORTED, "sector dimension >= 2^32");
    int L = 0;
    while (L < N && ipow(d, L + 1) <= kSpinMaxLow) ++L;
    const uint64_t nlo = ipow(d, L), H = ipow(d, N - L);
    if (H > kSpinMaxHigh) return fail(FTLM_EUNSUPPORTED, "high digit block beyond 2^27 labels");

    cudaStream_t stream = (cudaStream_t)stream_;
    ftlm_basis *b = new (std::nothrow) ftlm_basis();
    if (!b) return fail(FTLM_ENOMEM, "host allocation failed");
    b->N = N;
    b->K = A;
    b->two_sz = two_sz;
    b->two_s = two_s;
    b->key_n = N | (two_s << 8);
    b->D = D;
    b->mode = FTLM_RANK_CR;
    b->L = L;
    b->H = H;
    b->nblocks = 0;
    // N_nz of Eq. 10: per bond and ladder term, the states admitting the move
    uint64_t off = 0;
    for (int ai = 0; ai < two_s; ++ai)
        for (int aj = 1; aj <= two_s; ++aj) off += dims.at(N - 2, A - ai - aj);
    b->updates = D + 2ull * (uint64_t)n_bonds * off;
    const double s = 0.5 * two_s;
    double jabs = 0.0;
    for (int k = 0; k < n_bonds; ++k) jabs += std::fabs(J[k]);
    b->tau64 = 100.0 * 0x1p-53 * s * (s + 1.0) * jabs;  // ||S_i . S_j|| = s (s + 1)
    b->tau32 = 100.0 * 0x1p-24 * s * (s + 1.0) * jabs;
    cudaError_t ce = cudaGetDevice(&b->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (ce != cudaSuccess) {
        delete b;
        return cuda_fail(ce, "cudaGetDevice/cudaDeviceGetAttribute");
    }

    // Host tables: tlo/ulo over the d^L low labels grouped by digit sum, uoff the
    // group starts, thi[h] = sector labels below h d^L.
    const int amax_lo = L * two_s;
    std::vector<uint32_t> uoff(amax_lo + 2, 0);
    for (int a = 0; a <= amax_lo; ++a) uoff[a + 1] = uoff[a] + (uint32_t)dims.at(L, a);
    std::vector<uint16_t> tlo(nlo), ulo(nlo);
    {
        std::vector<uint32_t> fill(amax_lo + 1, 0);
        for (uint64_t l = 0; l < nlo; ++l) {
            int sum = 0;
            for (uint64_t m = l; m; m /= d) sum += (int)(m % d);
            tlo[l] = (uint16_t)fill[sum];
            ulo[uoff[sum] + fill[sum]] = (uint16_t)l;
            ++fill[sum];
        }
    }
    std::vector<uint32_t> thi(H);
    {
        uint64_t below = 0;
        for (uint64_t h = 0; h < H; ++h) {
            thi[h] = (uint32_t)below;
            int sum = 0;
            for (uint64_t m = h; m; m /= d) sum += (int)(m % d);
            below += dims.at(L, A - sum);
        }
    }
    // bonds: (i < j) positions, block flags, block-local powers; J and the ladder
    // factors.  Ordered by class -- both sites in the low block, both in the high
    // block, one in each (i low, j high, since i < j) -- so the kernels rank each
    // class with its own arithmetic.
    std::vector<uint4> slots(kMaxBondSlots, make_uint4(0, 0, 0, 0));
    std::vector<float> jf(kMaxBondSlots, 0.f);
    std::vector<double> jd(kMaxBondSlots, 0.0);
    uint32_t n_class[3] = {0, 0, 0};
    {
        int pos = 0;
        for (int cls = 0; cls < 3; ++cls)
            for (int k = 0; k < n_bonds; ++k) {
                const int i = std::min(bi[k], bj[k]), j = std::max(bi[k], bj[k]);
                const uint32_t hi_i = i >= L, hi_j = j >= L;
                const int c = hi_i ? 1 : (hi_j ? 2 : 0);
                if (c != cls) continue;
                slots[pos] = make_uint4((uint32_t)i | ((uint32_t)j << 8) | (hi_i << 16) | (hi_j << 17),
                                        (uint32_t)ipow(d, hi_i ? i - L : i), (uint32_t)ipow(d, hi_j ? j - L : j), 0u);
                jf[pos] = (float)J[k];
                jd[pos] = J[k];
                ++n_class[cls];
                ++pos;
            }
    }
    std::vector<float> upf(kSpinMaxTwoS + 1, 0.f);
    std::vector<double> upd(kSpinMaxTwoS + 1, 0.0);
    for (int a = 0; a < two_s; ++a) {
        const double m = a - s;
        upd[a] = std::sqrt(s * (s + 1.0) - m * (m + 1.0));
        upf[a] = (float)upd[a];
    }

    // One pooled block: small tables from one host image, then the coarse index.
    b->n_hs = ((D - 1) >> kHsShift) + 2;
    uint64_t offb = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = offb;
        offb = (offb + bytes + 255) & ~uint64_t(255);
        return o;
    };
    const uint64_t o_slots = take(slots.size() * sizeof(uint4));
    const uint64_t o_jf = take(jf.size() * sizeof(float));
    const uint64_t o_jd = take(jd.size() * sizeof(double));
    const uint64_t o_upf = take(upf.size() * sizeof(float));
    const uint64_t o_upd = take(upd.size() * sizeof(double));
    const uint64_t o_thi = take(H * sizeof(uint32_t));
    const uint64_t o_tlo = take(nlo * sizeof(uint16_t));
    const uint64_t o_ulo = take(nlo * sizeof(uint16_t));
    const uint64_t o_uoff = take(uoff.size() * sizeof(uint32_t));
    const uint64_t small_bytes = offb;
    const uint64_t o_hs = take(b->n_hs * sizeof(uint32_t));
    b->table_bytes = offb;
    std::vector<unsigned char> image(small_bytes, 0);
    std::memcpy(image.data() + o_slots, slots.data(), slots.size() * sizeof(uint4));
    std::memcpy(image.data() + o_jf, jf.data(), jf.size() * sizeof(float));
    std::memcpy(image.data() + o_jd, jd.data(), jd.size() * sizeof(double));
    std::memcpy(image.data() + o_upf, upf.data(), upf.size() * sizeof(float));
    std::memcpy(image.data() + o_upd, upd.data(), upd.size() * sizeof(double));
    std::memcpy(image.data() + o_thi, thi.data(), H * sizeof(uint32_t));
    std::memcpy(image.data() + o_tlo, tlo.data(), nlo * sizeof(uint16_t));
    std::memcpy(image.data() + o_ulo, ulo.data(), nlo * sizeof(uint16_t));
    std::memcpy(image.data() + o_uoff, uoff.data(), uoff.size() * sizeof(uint32_t));

    cudaMemPool_t pool = nullptr;
    cudaError_t e = table_pool(b->device, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&b->block, b->table_bytes, pool, stream);
    if (e != cudaSuccess) {
        delete b;
        return e == cudaErrorMemoryAllocation ? fail(FTLM_ENOMEM, "no device memory for the sector tables")
                                              : cuda_fail(e, "cudaMallocFromPoolAsync(spin tables)");
    }
    char *base = static_cast<char *>(b->block);
    b->thi = reinterpret_cast<uint32_t *>(base + o_thi);
    b->tlo = reinterpret_cast<uint16_t *>(base + o_tlo);
    b->ulo = reinterpret_cast<uint16_t *>(base + o_ulo);
    b->uoff = reinterpret_cast<uint32_t *>(base + o_uoff);
    b->hs = reinterpret_cast<uint32_t *>(base + o_hs);
    b->bond_slots = reinterpret_cast<uint4 *>(base + o_slots);
    b->basis = nullptr;
    b->clt = nullptr;
    SpinDev &p = b->spin;
    p.d = (uint32_t)d;
    p.two_s = (uint32_t)two_s;
    p.A = (uint32_t)A;
    p.nb = (uint32_t)n_bonds;
    p.n_ll = n_class[0];
    p.n_hh = n_class[1];
    // q = floor(n * ceil(2^k / d) / 2^k), k = 32 + ceil(log2 d): exact for n < 2^32
    // (Granlund & Montgomery 1994); the labels divided here are below 2^27.
    int lg = 0;
    while ((1 << lg) < d) ++lg;
    p.shift = 32u + (uint32_t)lg;
    p.magic = ((1ull << p.shift) + (uint64_t)d - 1) / (uint64_t)d;
    p.slots = b->bond_slots;
    p.jf = reinterpret_cast<const float *>(base + o_jf);
    p.jd = reinterpret_cast<const double *>(base + o_jd);
    p.upf = reinterpret_cast<const float *>(base + o_upf);
    p.upd = reinterpret_cast<const double *>(base + o_upd);
    // bond lists of the spin-1/2 kernels stay empty for this basis
    b->bonds_cr = BondList{};
    b->bonds_clt = BondList{};

    e = upload_async(base, image.data(), small_bytes, stream);
    if (e == cudaSuccess) {
        launch_hs_fill(b, stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && wait) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(b->block, stream);
        delete b;
        return cuda_fail(e, "spin sector table build");
    }
    *out = b;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_create_sectors(int N, int two_s, int n, const int *two_sz, int n_bonds,
                                                 const int *bi, const int *bj, const double *J, ftlm_rank_mode mode,
                                                 int wait, void *stream_, ftlm_basis **out)
{
    if (!out || !two_sz) return fail(FTLM_EINVAL, "NULL argument");
    if (n < 1 || n > FTLM_MAX_SECTORS) return fail(FTLM_EINVAL, "n out of range");
    for (int k = 0; k < n; ++k) out[k] = nullptr;
    cudaStream_t stream = (cudaStream_t)stream_;
    ftlm_status st = FTLM_OK;
    for (int k = 0; k < n && st == FTLM_OK; ++k)
        st = two_s == 1 ? basis_create_half(N, two_sz[k], n_bonds, bi, bj, J, mode, stream, false, &out[k])
                        : basis_create_spin(N, two_s, two_sz[k], n_bonds, bi, bj, J, stream, false, &out[k]);
    if (st == FTLM_OK && wait) {
        const cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) st = cuda_fail(e, "sector table build");
    }
    if (st != FTLM_OK) {  // keeps the first error's message; frees in stream order
        for (int k = 0; k < n; ++k) {
            ftlm_basis_destroy_async(out[k], stream_);
            out[k] = nullptr;
        }
    }
    return st;
}
