// Sector setup (step a1): validation, digit-block rank tables, the CLT arrays and
// the sorted basis, plus the rank/label entry points used to check them.
//
// Combinatorial rank at s = 1/2 (Eq. 15-17, Algorithm 1).  For s = 1/2 the table
// D(m, A) of Eq. 15 is Pascal's triangle, D(m, A) = C(m, A), and the cumulative
// table of Eq. 16 reduces to D_c(p, A, 1) = C(p, A), D_c(p, A, 0) = 0.  Algorithm 1
// walks the digits p = N-1 .. 0 with A starting at A_tot = K (Eq. 17) and adds
// C(p, A) at every set bit before decrementing A; equivalently the k-th set bit
// from the bottom, at position p_k, contributes C(p_k, k).
//
// The paper's first GPU adaptation replaces the per-digit inner scan by one table
// lookup per digit.  The library takes the same step for a whole block of digits:
// split the label n into a low block l (the L lowest bits) and a high block h.
// The contributions of the low bits depend only on l (their k counts only bits
// below them): tlo[l].  The contributions of the high bits depend on h and on the
// number of low set bits, which inside a sector is K - popcount(h): thi[h].  So
//     rank(n) = thi[n >> L] + tlo[n & (2^L - 1)],
// two lookups instead of N digit steps, bit-identical to Algorithm 1.  thi[h] is
// also the number of sector labels below h * 2^L (it is defined that way for every
// h, which keeps thi non-decreasing and lets the inverse map binary-search it).
//
// CLT (Eq. 18-21): blocks of 32 labels with occupancy mask M_b and prefix count
// C_b.  At s = 1/2 the mask of block b depends only on popcount(b): label 32b + j
// is in the sector iff popcount(j) = K - popcount(b); and C_b is the number of
// sector labels below 32 b.  Both are computed per block in parallel; the result
// is bit-identical to the paper's single pass over the basis plus cumulative
// popcount sum.  M_b and C_b are stored interleaved, one 8-byte entry per block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ftlm_internal.cuh"

namespace ftlm {

namespace {

uint64_t g_binom[65][65];
std::once_flag g_binom_once;

void init_binom()
{
    std::call_once(g_binom_once, [] {
        for (int n = 0; n <= 64; ++n)
            for (int k = 0; k <= 64; ++k)
                g_binom[n][k] = (k == 0) ? 1 : (n == 0 ? 0 : g_binom[n - 1][k - 1] + g_binom[n - 1][k]);
    });
}

uint64_t binom(int n, int k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    return g_binom[n][k];
}

// Number of N-bit labels below v with K set bits.
uint64_t count_below(uint64_t v, int N, int K)
{
    uint64_t cnt = 0;
    int above = 0;
    for (int p = N - 1; p >= 0; --p) {
        if ((v >> p) & 1u) {
            cnt += binom(p, K - above);
            ++above;
        }
    }
    return cnt;
}

int popc64(uint64_t v) { return __builtin_popcountll(v); }

// ---- device kernels ---------------------------------------------------------

// Inverse map t -> label through the digit-block tables: h is the last high
// pattern with thi[h] <= t (thi is non-decreasing; the one found has room for t),
// then the low pattern is entry t - thi[h] of popcount group K - popcount(h).
__device__ __forceinline__ uint64_t unrank_label(uint32_t t, const SectorTables &s)
{
    uint32_t lo = 0, hi = s.H;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(s.thi + mid) <= t) lo = mid;
        else hi = mid;
    }
    uint32_t r_lo = t - __ldg(s.thi + lo);
    int c = s.K - __popc(lo);
    uint32_t l = __ldg(s.ulo + __ldg(s.uoff + c) + r_lo);
    return ((uint64_t)lo << s.L) | l;
}

// hs[k] = high pattern of row min(k << kHsShift, D - 1).
__global__ void hs_fill_kernel(SectorTables s, uint64_t n_hs, uint32_t *hs)
{
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_hs;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t row = k << kHsShift;
        const uint32_t t = (uint32_t)(row < s.D ? row : s.D - 1);
        uint32_t lo = 0, hi = s.H;
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (__ldg(s.thi + mid) <= t) lo = mid;
            else hi = mid;
        }
        hs[k] = lo;
    }
}

__global__ void basis_fill_kernel(SectorTables s, uint32_t *basis)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < s.D;
         t += (uint64_t)gridDim.x * blockDim.x)
        basis[t] = (uint32_t)unrank_label((uint32_t)t, s);
}

// CLT entry of block b: occupancy mask and count of sector labels below 32 b.
__global__ void clt_fill_kernel(int N, int K, uint64_t nblocks, const uint64_t *binom_g, uint2 *clt)
{
    __shared__ uint64_t sb[33 * 33];
    for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) sb[i] = binom_g[i];
    __syncthreads();
    const int wbits = N < 5 ? N : 5;  // label bits inside a block
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        int c = K - __popcll(b);
        uint32_t mask = 0;
        if (c >= 0 && c <= wbits)
            for (int j = 0; j < (1 << wbits); ++j)
                if (__popc(j) == c) mask |= 1u << j;
        // count_below(32 b): walk the set bits of b (label bits 5 ..) from the top
        uint64_t cnt = 0;
        int above = 0;
        for (int p = N - 1; p >= 5; --p) {
            if ((b >> (p - 5)) & 1u) {
                int k = K - above;
                if (k >= 0 && k <= p) cnt += sb[p * 33 + k];
                ++above;
            }
        }
        clt[b] = make_uint2(mask, (uint32_t)cnt);
    }
}

__global__ void labels_kernel(SectorTables s, int clt_mode, uint64_t first, uint64_t count,
                              uint64_t *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t t = (uint32_t)(first + i);
        out[i] = clt_mode ? (uint64_t)__ldg(s.basis + t) : unrank_label(t, s);
    }
}

__global__ void rank_kernel(SectorTables s, int clt_mode, uint64_t count, const uint64_t *labels,
                            int64_t *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t n = labels[i];
        int64_t r = -1;
        if ((n >> s.N) == 0 && __popcll(n) == s.K) {
            if (clt_mode) {
                // Algorithm 2 / Eq. 19-20
                uint2 e = __ldg(s.clt + (n >> 5));
                uint32_t j = (uint32_t)(n & 31u);
                if ((e.x >> j) & 1u) r = (int64_t)e.y + __popc(e.x & ((1u << j) - 1u));
            } else {
                r = (int64_t)__ldg(s.thi + (n >> s.L)) + __ldg(s.tlo + (n & s.lomask));
            }
        }
        out[i] = r;
    }
}

__global__ void clt_split_kernel(const uint2 *clt, uint64_t nblocks, uint32_t *mask, uint32_t *prefix)
{
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nblocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        uint2 e = clt[b];
        mask[b] = e.x;
        prefix[b] = e.y;
    }
}

int grid_for(uint64_t n, int threads, int num_sms)
{
    uint64_t g = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms * 16;
    return (int)std::max<uint64_t>(1, std::min(g, cap));
}

uint64_t align256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

}  // namespace

int max_row_grid(const ftlm_basis *b) { return b->num_sms * kMaxBlocksPerSm; }

bool build_hi_walk(const ftlm_basis *b, int rh, HiWalk *w)
{
    if (b->two_s != 1 || b->mode != FTLM_RANK_CR || !b->uhi) return false;
    if (b->N <= b->L || b->n_hi_bonds < 1 || b->n_hi_bonds > kMaxHiBonds) return false;
    if (rh < 1 || rh > 32) return false;
    init_binom();
    const int nhb = b->N - b->L;
    HiWalk h{};
    h.nbonds = b->n_hi_bonds;
    h.rh = rh;
    h.jsum4 = b->jsum4_hi;
    h.uhi = b->uhi;
    h.bonds = b->bond_slots + 6 * kMaxBondSlots;
    uint64_t tiles = 0;
    for (int q = 0; q <= b->L; ++q) {
        const int p = b->K - q;
        if (p < 0 || p > nhb) continue;
        const uint64_t nl = binom(b->L, q), nh = binom(nhb, p);
        if (!nl || !nh) continue;
        const int g = h.ngroups++;
        h.tile0[g] = (uint32_t)tiles;
        h.nl[g] = (uint32_t)nl;
        h.nh[g] = (uint32_t)nh;
        h.hoff[g] = b->uhi_off[p];
        h.nr[g] = (uint32_t)((nh + rh - 1) / rh);
        tiles += ((nl + 31) / 32) * h.nr[g];
    }
    if (tiles >= (1ull << 32)) return false;
    h.tile0[h.ngroups] = (uint32_t)tiles;
    h.ntiles = (uint32_t)tiles;
    *w = h;
    return true;
}

bool build_lo_walk(const ftlm_basis *b, LoWalk *w)
{
    if (b->two_s != 1 || b->mode != FTLM_RANK_CR || !b->lo_tiles || !b->n_lo_tiles) return false;
    LoWalk a{};
    a.ntiles = b->n_lo_tiles;
    a.n_ll = b->n_ll_a;
    a.n_cr = b->n_cr_a;
    a.nb = a.n_ll + a.n_cr;
    a.jsum4 = b->jsum4_a;
    for (int p = 0; p <= kMaxHighBits; ++p) a.hend[p] = b->uhi_off[p + 1];
    a.hend[kMaxHighBits + 1] = b->uhi_off[kMaxHighBits + 1];
    a.tiles = b->lo_tiles;
    a.uhi = b->uhi;
    a.slots_f32 = b->bond_slots + 4 * kMaxBondSlots;
    a.slots_f64 = b->bond_slots + 5 * kMaxBondSlots;
    *w = a;
    return true;
}

void launch_hs_fill(const ftlm_basis *b, cudaStream_t stream)
{
    hs_fill_kernel<<<grid_for(b->n_hs, 256, b->num_sms), 256, 0, stream>>>(b->tables(), b->n_hs, b->hs);
    note_launch();
}

int row_grid(const ftlm_basis *b, uint64_t rows, int occ)
{
    occ = std::max(1, std::min(occ, kMaxBlocksPerSm));
    uint64_t need = (rows + kRowThreads - 1) / kRowThreads;
    uint64_t cap = (uint64_t)b->num_sms * occ;
    return (int)std::max<uint64_t>(1, std::min(need, cap));
}

}  // namespace ftlm

using namespace ftlm;

ftlm::SectorTables ftlm_basis::tables() const
{
    SectorTables s;
    s.D = (uint32_t)D;
    s.N = N;
    s.K = K;
    s.L = L;
    if (two_s > 1) {  // base-d digit blocks: lomask + 1 = d^L low labels
        uint32_t nlo = 1;
        for (int k = 0; k < L; ++k) nlo *= (uint32_t)(two_s + 1);
        s.lomask = nlo - 1u;
    } else {
        s.lomask = (1u << L) - 1u;
    }
    s.H = (uint32_t)H;
    s.thi = thi;
    s.tlo = tlo;
    s.ulo = ulo;
    s.uoff = uoff;
    s.hs = hs;
    s.basis = basis;
    s.clt = clt;
    return s;
}

extern "C" ftlm_status ftlm_basis_create(int N, int two_sz, int n_bonds, const int *bi,
                                         const int *bj, const double *J, ftlm_rank_mode mode,
                                         void *stream_, ftlm_basis **out)
{
    return ftlm::basis_create_half(N, two_sz, n_bonds, bi, bj, J, mode, (cudaStream_t)stream_, true, out);
}

// wait: return once the tables are built (else once their build is queued).
ftlm_status ftlm::basis_create_half(int N, int two_sz, int n_bonds, const int *bi, const int *bj, const double *J,
                                    ftlm_rank_mode mode, cudaStream_t stream_, bool wait, ftlm_basis **out)
{
    if (!out) return fail(FTLM_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > FTLM_MAX_SITES) return fail(FTLM_EINVAL, "N out of range");
    if (two_sz < -N || two_sz > N || ((two_sz + N) & 1)) return fail(FTLM_EINVAL, "bad two_sz");
    if (n_bonds < 0) return fail(FTLM_EINVAL, "n_bonds < 0");
    if (n_bonds > FTLM_MAX_BONDS) return fail(FTLM_EUNSUPPORTED, "more than FTLM_MAX_BONDS bonds");
    if (n_bonds > 0 && (!bi || !bj || !J)) return fail(FTLM_EINVAL, "bond arrays are NULL");
    if (mode != FTLM_RANK_AUTO && mode != FTLM_RANK_CLT && mode != FTLM_RANK_CR)
        return fail(FTLM_EINVAL, "bad rank mode");
    std::vector<std::pair<int, int>> seen;
    for (int b = 0; b < n_bonds; ++b) {
        int i = std::min(bi[b], bj[b]), j = std::max(bi[b], bj[b]);
        if (i < 0 || j >= N) return fail(FTLM_EINVAL, "bond site out of range");
        if (i == j) return fail(FTLM_EINVAL, "bond joins a site to itself");
        if (!(J[b] == J[b]) || J[b] - J[b] != 0.0) return fail(FTLM_EINVAL, "non-finite coupling");
        seen.emplace_back(i, j);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return fail(FTLM_EINVAL, "duplicate bond");

    init_binom();
    const int K = (N + two_sz) / 2;
    const uint64_t D = binom(N, K);
    if (D >= (1ull << 32)) return fail(FTLM_EUNSUPPORTED, "sector dimension >= 2^32");
    if (mode == FTLM_RANK_AUTO) {
        // Measured on GB300 with blocks of chains: combinatorial ranking is the faster
        // map from 2^20 rows up (its Lanczos H.v launches take rows in dynamic order,
        // whose gathers share L2; 13 % faster on the N = 30 icosahedral sector), CLT
        // below (many small sectors of a batch, where CR restages its rank table per
        // sector).  CLT also needs its tables (basis array + Eq. 21) to fit in a
        // quarter of the device memory.
        mode = FTLM_RANK_CR;
        size_t free_b = 0, total_b = 0;
        if (N <= 32 && D < kAutoCrRows && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const uint64_t clt_bytes = 4 * D + 8 * (((1ull << N) + 31) / 32);
            if (clt_bytes <= total_b / 4) mode = FTLM_RANK_CLT;
        }
    }
    if (mode == FTLM_RANK_CLT && N > 32) return fail(FTLM_EUNSUPPORTED, "CLT needs N <= 32");

    cudaStream_t stream = (cudaStream_t)stream_;
    ftlm_basis *b = new (std::nothrow) ftlm_basis();
    if (!b) return fail(FTLM_ENOMEM, "host allocation failed");
    b->N = N;
    b->K = K;
    b->two_sz = two_sz;
    b->two_s = 1;
    b->key_n = N;
    b->D = D;
    b->mode = mode;
    b->L = std::min(N, kLoBitsMax);
    b->H = 1ull << (N - b->L);
    b->nblocks = ((1ull << N) + 31) / 32;
    b->updates = D + 2ull * (uint64_t)n_bonds * binom(N - 2, K - 1);
    double jabs = 0.0;
    for (int k = 0; k < n_bonds; ++k) jabs += std::fabs(J[k]);
    b->tau64 = 100.0 * 0x1p-53 * 0.75 * jabs;
    b->tau32 = 100.0 * 0x1p-24 * 0.75 * jabs;
    cudaError_t ce = cudaGetDevice(&b->device);
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (ce != cudaSuccess) {
        delete b;
        return cuda_fail(ce, "cudaGetDevice/cudaDeviceGetAttribute");
    }

    // Bond lists: CLT keeps the caller's order; CR groups by low/high block.  Both
    // are padded to whole chunks with dummy bonds (mask 0, coupling 0).
    const int L = b->L;
    double jsum4 = 0.0;
    for (int k = 0; k < n_bonds; ++k) jsum4 += J[k] / 4.0;
    auto round_up = [](int v) { return (v + kBondChunk - 1) / kBondChunk * kBondChunk; };
    // host images of the slot arrays: CR, CLT and walk A (FP32 and FP64 each), walk B
    std::vector<uint4> slots(7 * (size_t)kMaxBondSlots, make_uint4(0u, 0u, 0u, 0u));
    auto put = [&](int which, int pos, uint32_t mlo, uint32_t mhi, double jh) {
        float f = (float)jh;
        uint32_t fb;
        std::memcpy(&fb, &f, 4);
        uint64_t db;
        std::memcpy(&db, &jh, 8);
        slots[(size_t)(2 * which) * kMaxBondSlots + pos] = make_uint4(mlo, mhi, fb, 0u);
        slots[(size_t)(2 * which + 1) * kMaxBondSlots + pos] =
            make_uint4(mlo, mhi, (uint32_t)db, (uint32_t)(db >> 32));
    };
    {
        BondList &c = b->bonds_cr;
        std::vector<int> lo, hi, rest;
        for (int k = 0; k < n_bonds; ++k) {
            bool il = bi[k] < L, jl = bj[k] < L;
            (il && jl ? lo : (!il && !jl) ? hi : rest).push_back(k);
        }
        const int nlo = (int)lo.size() / kBondChunk * kBondChunk;
        const int nhi = (int)hi.size() / kBondChunk * kBondChunk;
        std::vector<int> order(lo.begin(), lo.begin() + nlo);
        order.insert(order.end(), hi.begin(), hi.begin() + nhi);
        order.insert(order.end(), lo.begin() + nlo, lo.end());
        order.insert(order.end(), hi.begin() + nhi, hi.end());
        order.insert(order.end(), rest.begin(), rest.end());
        for (int pos = 0; pos < (int)order.size(); ++pos) {
            const int k = order[pos];
            const uint64_t m = (1ull << bi[k]) | (1ull << bj[k]);
            if (pos < nlo) put(0, pos, (uint32_t)m, 0u, J[k] / 2.0);
            else if (pos < nlo + nhi) put(0, pos, 0u, (uint32_t)(m >> L), J[k] / 2.0);
            else put(0, pos, (uint32_t)m, (uint32_t)(m >> 32), J[k] / 2.0);
        }
        c.n_lo = nlo;
        c.n_hi = nhi;
        c.nb = nlo + nhi + round_up(n_bonds - nlo - nhi);
        c.jsum4 = jsum4;
    }
    {
        // split H.v: walk A (walka.cu) takes the lo-lo bonds as low masks, then the
        // cross bonds as {2^i, 2^(j-L)}, each list padded to a multiple of 4 slots;
        // walk B the high-high bonds as one compact list
        std::vector<int> lo, hi, rest;
        for (int k = 0; k < n_bonds; ++k) {
            bool il = bi[k] < L, jl = bj[k] < L;
            (il && jl ? lo : (!il && !jl) ? hi : rest).push_back(k);
        }
        int pos = 0;
        double j4 = 0.0;
        auto put_a = [&](uint32_t x, uint32_t y, double jh) {
            const float f = (float)jh;
            uint32_t fb;
            std::memcpy(&fb, &f, 4);
            uint64_t db;
            std::memcpy(&db, &jh, 8);
            slots[(size_t)4 * kMaxBondSlots + pos] = make_uint4(x, y, fb, 0u);
            slots[(size_t)5 * kMaxBondSlots + pos] = make_uint4(x, y, (uint32_t)db, (uint32_t)(db >> 32));
            ++pos;
            j4 += jh / 2.0;
        };
        for (int k : lo) put_a((1u << bi[k]) | (1u << bj[k]), 0u, J[k] / 2.0);
        b->n_ll_a = (int)(lo.size() + 3) / 4 * 4;
        pos = b->n_ll_a;
        for (int k : rest) {
            const int i = std::min(bi[k], bj[k]), j = std::max(bi[k], bj[k]);
            put_a(1u << i, 1u << (j - L), J[k] / 2.0);
        }
        b->n_cr_a = (int)(rest.size() + 3) / 4 * 4;
        b->jsum4_a = j4;
        b->n_hi_bonds = (int)hi.size();
        double jh4 = 0.0;
        for (int pos = 0; pos < (int)hi.size() && pos < kMaxBondSlots; ++pos) {
            const int k = hi[pos];
            const double jh = J[k] / 2.0;
            const float f = (float)jh;
            uint32_t fb;
            std::memcpy(&fb, &f, 4);
            uint64_t db;
            std::memcpy(&db, &jh, 8);
            const uint64_t m = ((1ull << bi[k]) | (1ull << bj[k])) >> L;
            slots[(size_t)6 * kMaxBondSlots + pos] = make_uint4((uint32_t)m, fb, (uint32_t)db, (uint32_t)(db >> 32));
            jh4 += J[k] / 4.0;
        }
        b->jsum4_hi = jh4;
    }
    {
        BondList &c = b->bonds_clt;
        for (int k = 0; k < n_bonds; ++k) {
            const uint64_t m = (1ull << bi[k]) | (1ull << bj[k]);
            put(1, k, (uint32_t)m, (uint32_t)(m >> 32), J[k] / 2.0);
        }
        c.n_lo = c.n_hi = 0;
        c.nb = round_up(n_bonds);
        c.jsum4 = jsum4;
    }

    // Digit-block tables on the host.
    const uint32_t nlo = 1u << L;
    std::vector<uint16_t> tlo(nlo), ulo(nlo);
    std::vector<uint32_t> thi(b->H);
    {
        uint32_t off = 0;
        for (int c = 0; c <= kLoBitsMax + 1; ++c) {
            b->ulo_off[c] = off;
            if (c <= L) off += (uint32_t)binom(L, c);
        }
        for (uint32_t v = 0; v < nlo; ++v) {
            uint64_t r = 0;
            int k = 0;
            for (int p = 0; p < L; ++p)
                if ((v >> p) & 1u) r += binom(p, ++k);
            tlo[v] = (uint16_t)r;
            ulo[b->ulo_off[popc64(v)] + r] = (uint16_t)v;
        }
        for (uint64_t h = 0; h < b->H; ++h) thi[h] = (uint32_t)count_below(h << L, N, K);
    }
    // High patterns grouped by popcount, ascending (walk B of the split H.v).
    std::vector<uint32_t> uhi(b->H);
    {
        const int nh = N - L;
        uint32_t off = 0;
        for (int p = 0; p <= kMaxHighBits + 1; ++p) {
            b->uhi_off[p] = off;
            if (p <= nh) off += (uint32_t)binom(nh, p);
        }
        std::vector<uint32_t> fill(b->uhi_off, b->uhi_off + kMaxHighBits + 2);
        for (uint64_t h = 0; h < b->H; ++h) uhi[fill[popc64(h)]++] = (uint32_t)h;
    }

    // Tile table of the blocked walk A (LoWalk), for sectors that can run the split:
    // the runs of kLoRun high patterns of one popcount class in the order of their
    // first pattern, each followed by its column chunks.
    std::vector<uint32_t> lo_tiles;
    if (mode == FTLM_RANK_CR && N > L && b->n_hi_bonds >= 1 && b->n_hi_bonds <= kMaxHiBonds) {
        const int nh = N - L;
        std::vector<uint32_t> cnt(nh + 1, 0u);
        for (uint64_t h = 0; h < b->H; ++h) {
            const int p = popc64(h);
            const uint32_t idx = cnt[p]++;
            const int q = K - p;
            if (idx % kLoRun || q < 0 || q > L) continue;
            const uint32_t nch = (uint32_t)((binom(L, q) + 31) / 32);
            const uint32_t pos = b->uhi_off[p] + idx;
            for (uint32_t c = 0; c < nch; ++c) lo_tiles.push_back(pos << 7 | c);
        }
    }
    b->n_lo_tiles = (uint32_t)lo_tiles.size();

    // One stream-ordered allocation holds every table: the small ones first (bond
    // slots, thi, tlo, ulo, uoff, and the binomials the CLT build reads), filled by
    // one copy from a host image, then the coarse index and, for CLT, the basis
    // array and the CLT entries, which kernels fill on the device.
    b->n_hs = ((D - 1) >> kHsShift) + 2;
    const bool clt = mode == FTLM_RANK_CLT;
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const uint64_t o_slots = take(slots.size() * sizeof(uint4));
    const uint64_t o_thi = take(b->H * sizeof(uint32_t));
    const uint64_t o_tlo = take(nlo * sizeof(uint16_t));
    const uint64_t o_ulo = take(nlo * sizeof(uint16_t));
    const uint64_t o_uoff = take(sizeof(b->ulo_off));
    const uint64_t o_uhi = take(b->H * sizeof(uint32_t));
    const uint64_t o_lot = take(lo_tiles.size() * sizeof(uint32_t));
    const uint64_t o_binom = clt ? take(33 * 33 * sizeof(uint64_t)) : off;
    const uint64_t small_bytes = off;
    const uint64_t o_hs = take(b->n_hs * sizeof(uint32_t));
    const uint64_t o_basis = clt ? take(D * sizeof(uint32_t)) : off;
    const uint64_t o_clt = clt ? take(b->nblocks * sizeof(uint2)) : off;
    b->table_bytes = off;

    std::vector<unsigned char> image(small_bytes, 0);
    std::memcpy(image.data() + o_slots, slots.data(), slots.size() * sizeof(uint4));
    std::memcpy(image.data() + o_thi, thi.data(), b->H * sizeof(uint32_t));
    std::memcpy(image.data() + o_tlo, tlo.data(), nlo * sizeof(uint16_t));
    std::memcpy(image.data() + o_ulo, ulo.data(), nlo * sizeof(uint16_t));
    std::memcpy(image.data() + o_uoff, b->ulo_off, sizeof(b->ulo_off));
    std::memcpy(image.data() + o_uhi, uhi.data(), b->H * sizeof(uint32_t));
    if (!lo_tiles.empty()) std::memcpy(image.data() + o_lot, lo_tiles.data(), lo_tiles.size() * sizeof(uint32_t));
    if (clt) {
        uint64_t *bh = reinterpret_cast<uint64_t *>(image.data() + o_binom);
        for (int n = 0; n <= 32; ++n)
            for (int k = 0; k <= 32; ++k) bh[n * 33 + k] = binom(n, k);
    }

    cudaMemPool_t pool = nullptr;
    cudaError_t e = table_pool(b->device, &pool);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "table memory pool");
    }
    e = cudaMallocFromPoolAsync(&b->block, b->table_bytes, pool, stream);
    if (e != cudaSuccess) {
        delete b;
        return e == cudaErrorMemoryAllocation ? fail(FTLM_ENOMEM, "no device memory for the sector tables")
                                              : cuda_fail(e, "cudaMallocFromPoolAsync(tables)");
    }
    char *base = static_cast<char *>(b->block);
    b->bond_slots = reinterpret_cast<uint4 *>(base + o_slots);
    b->thi = reinterpret_cast<uint32_t *>(base + o_thi);
    b->tlo = reinterpret_cast<uint16_t *>(base + o_tlo);
    b->ulo = reinterpret_cast<uint16_t *>(base + o_ulo);
    b->uoff = reinterpret_cast<uint32_t *>(base + o_uoff);
    b->uhi = reinterpret_cast<uint32_t *>(base + o_uhi);
    b->lo_tiles = lo_tiles.empty() ? nullptr : reinterpret_cast<uint32_t *>(base + o_lot);
    b->hs = reinterpret_cast<uint32_t *>(base + o_hs);
    b->basis = clt ? reinterpret_cast<uint32_t *>(base + o_basis) : nullptr;
    b->clt = clt ? reinterpret_cast<uint2 *>(base + o_clt) : nullptr;
    b->bonds_cr.slots_f32 = b->bond_slots;
    b->bonds_cr.slots_f64 = b->bond_slots + kMaxBondSlots;
    b->bonds_clt.slots_f32 = b->bond_slots + 2 * kMaxBondSlots;
    b->bonds_clt.slots_f64 = b->bond_slots + 3 * kMaxBondSlots;

    // The copy returns once the image is staged, so `image` may go out of scope;
    // the kernels below follow it in stream order.
    e = upload_async(base, image.data(), small_bytes, stream);
    if (e == cudaSuccess) {
        launch_hs_fill(b, stream);
        if (clt) {
            const uint64_t *binom_d = reinterpret_cast<const uint64_t *>(base + o_binom);
            basis_fill_kernel<<<grid_for(D, 256, b->num_sms), 256, 0, stream>>>(b->tables(), b->basis);
            note_launch();
            clt_fill_kernel<<<grid_for(b->nblocks, 256, b->num_sms), 256, 0, stream>>>(N, K, b->nblocks, binom_d,
                                                                                        b->clt);
            note_launch();
        }
        e = cudaGetLastError();
    }
    // With wait, the tables are complete when create returns (only this stream is
    // waited for).
    if (e == cudaSuccess && wait) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(b->block, stream);
        delete b;
        return cuda_fail(e, "sector table build");
    }
    *out = b;
    return FTLM_OK;
}

extern "C" void ftlm_basis_destroy(ftlm_basis *b)
{
    if (!b) return;
    // Wait for every queued kernel (any of them may read the tables), then return
    // the block to the pool.
    cudaDeviceSynchronize();
    cudaFreeAsync(b->block, 0);
    delete b;
}

extern "C" ftlm_status ftlm_basis_destroy_async(ftlm_basis *b, void *stream)
{
    if (!b) return FTLM_OK;
    const cudaError_t e = cudaFreeAsync(b->block, (cudaStream_t)stream);
    delete b;
    return e == cudaSuccess ? FTLM_OK : cuda_fail(e, "cudaFreeAsync(tables)");
}

extern "C" ftlm_status ftlm_basis_set_schedule(ftlm_basis *b, ftlm_hv_schedule schedule, int rows_per_tile)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (schedule != FTLM_HV_AUTO && schedule != FTLM_HV_ONE_WALK && schedule != FTLM_HV_SPLIT)
        return fail(FTLM_EINVAL, "bad H.v schedule");
    if (rows_per_tile < 0 || rows_per_tile > 32) return fail(FTLM_EINVAL, "rows_per_tile must be 0..32");
    b->hv_schedule = schedule;
    b->walk_rh = rows_per_tile;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_dim(const ftlm_basis *b, uint64_t *dim)
{
    if (!b || !dim) return fail(FTLM_EINVAL, "NULL argument");
    *dim = b->D;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_bytes(const ftlm_basis *b, uint64_t *bytes)
{
    if (!b || !bytes) return fail(FTLM_EINVAL, "NULL argument");
    *bytes = b->table_bytes;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_mode(const ftlm_basis *b, ftlm_rank_mode *mode)
{
    if (!b || !mode) return fail(FTLM_EINVAL, "NULL argument");
    *mode = b->mode;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_updates(const ftlm_basis *b, uint64_t *updates)
{
    if (!b || !updates) return fail(FTLM_EINVAL, "NULL argument");
    *updates = b->updates;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_labels(const ftlm_basis *b, uint64_t first, uint64_t count,
                                         uint64_t *labels_dev, void *stream)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (first > b->D || count > b->D - first) return fail(FTLM_EINVAL, "index range beyond D");
    if (count == 0) return FTLM_OK;
    if (!labels_dev) return fail(FTLM_EINVAL, "labels_dev is NULL");
    if (b->two_s > 1) return launch_spin_labels(b, first, count, labels_dev, (cudaStream_t)stream);
    labels_kernel<<<grid_for(count, 256, b->num_sms), 256, 0, (cudaStream_t)stream>>>(
        b->tables(), b->mode == FTLM_RANK_CLT, first, count, labels_dev);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_rank(const ftlm_basis *b, uint64_t count, const uint64_t *labels_dev,
                                       int64_t *index_dev, void *stream)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (count == 0) return FTLM_OK;
    if (!labels_dev || !index_dev) return fail(FTLM_EINVAL, "NULL device pointer");
    if (b->two_s > 1) return launch_spin_rank(b, count, labels_dev, index_dev, (cudaStream_t)stream);
    rank_kernel<<<grid_for(count, 256, b->num_sms), 256, 0, (cudaStream_t)stream>>>(
        b->tables(), b->mode == FTLM_RANK_CLT, count, labels_dev, index_dev);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_basis_clt(const ftlm_basis *b, uint32_t *mask_dev, uint32_t *prefix_dev,
                                      void *stream)
{
    if (!b) return fail(FTLM_EINVAL, "NULL basis");
    if (b->mode != FTLM_RANK_CLT) return fail(FTLM_EUNSUPPORTED, "basis has no CLT (CR mode)");
    if (!mask_dev || !prefix_dev) return fail(FTLM_EINVAL, "NULL device pointer");
    clt_split_kernel<<<grid_for(b->nblocks, 256, b->num_sms), 256, 0, (cudaStream_t)stream>>>(
        b->clt, b->nblocks, mask_dev, prefix_dev);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}
