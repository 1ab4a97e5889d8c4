// Walk A of the split Lanczos H.v (CR, spin 1/2) with the rows of a block staged in
// shared memory: the low-low and cross bonds of Eq. 12-14 in label order.
//
// Rows (h, l) of one high pattern h form a contiguous group of C(L, c) rows,
// c = K - popcount(h), in ascending order of l.  A low-low bond changes l only and
// keeps its popcount, so its source row lies in the same group; if the bond also
// leaves the top S bits of l alone, the source lies in the same block of rows with
// equal top bits (a contiguous run of C(L - S, c - popcount(top)) rows).  A CTA
// claims such a block from a counter, copies its x rows into shared memory, and
// serves every gather that lands inside the block from there; the other gathers
// (cross bonds, low-low bonds on the top S bits) read global memory.  S is the
// smallest split that fits the largest block in kStageBytes, e.g. S = 1 for rows of
// 32 bytes at L = 14 (1716 rows, 54 KB).  The staged rows also give the row's own
// x[t] for the diagonal term.  In L2 these gathers would move about a third of the
// gather traffic of a step, which is what bounds the H.v (its L2 read rate).
//
// Blocks are claimed in label order (h, then top bits), so the grid walks the rows
// like the one-walk kernel and the cross-bond sources stay in a narrow, L2-resident
// window.  The epilogue is walk A's (no alpha): y = (H_A u_j) / s_j - c u_{j-1}.
#include <algorithm>

#include "epi.cuh"
#include "ftlm_internal.cuh"
#include "reduce.cuh"
#include "rows.cuh"
#include "vec.cuh"

namespace ftlm {

namespace {

constexpr int kStageThreads = 256;
constexpr size_t kStageBytes = 56 * 1024;  // staged x rows per CTA (two CTAs per SM)

// B values of one staged row (16-byte vector loads where the row allows).
template <int B> __device__ __forceinline__ void ld_row_smem(const float *p, float (&v)[B])
{
    if constexpr (B % 4 == 0) {
#pragma unroll
        for (int i = 0; i < B / 4; ++i) {
            const float4 f = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = f.x, v[4 * i + 1] = f.y, v[4 * i + 2] = f.z, v[4 * i + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) v[i] = p[i];
    }
}
template <int B> __device__ __forceinline__ void ld_row_smem(const double *p, double (&v)[B])
{
    if constexpr (B % 2 == 0) {
#pragma unroll
        for (int i = 0; i < B / 2; ++i) {
            const double2 d = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = d.x, v[2 * i + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) v[i] = p[i];
    }
}

struct StagedWalk {
    uint32_t nblocks;  // H << S blocks (h, top bits), many of them empty
    int S;             // top low bits that split a group into blocks
    uint32_t cap;      // rows of the largest block
};

template <typename V, int B, int C>
__global__ void __launch_bounds__(kStageThreads, 2)
walk_a_staged_kernel(const SectorTables s, const BondList bl, const StagedWalk w, const V *__restrict__ x, V *y,
                     const EpiDev ep)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // [staged rows: cap x B values][tlo: 2^L u16]
    V *s_x = reinterpret_cast<V *>(smem);
    uint16_t *s_tlo = reinterpret_cast<uint16_t *>(smem + (size_t)w.cap * B * sizeof(V));
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ V s_inv_s[B], s_c_prev[B];
    __shared__ uint32_t s_binom[kLoBitsMax + 1][kLoBitsMax + 1];
    __shared__ uint32_t s_cur, s_next;
    if (epi_begin<V, B>(ep, s_inv_s, s_c_prev)) return;
    {
        const uint4 *src = sizeof(V) == 4 ? bl.slots_f32 : bl.slots_f64;
        for (int i = threadIdx.x; i < bl.nb; i += blockDim.x) s_bond[i] = src[i];
    }
    for (uint32_t i = threadIdx.x; i <= s.lomask; i += blockDim.x) s_tlo[i] = __ldg(s.tlo + i);
    for (int i = threadIdx.x; i < (kLoBitsMax + 1) * (kLoBitsMax + 1); i += blockDim.x) {
        const int n = i / (kLoBitsMax + 1), k = i % (kLoBitsMax + 1);
        uint32_t c = 0;  // C(n, k) by the multiplicative formula (exact in 32 bits for n <= 14)
        if (k <= n) {
            c = 1;
            for (int j = 1; j <= k; ++j) c = c * (uint32_t)(n - k + j) / (uint32_t)j;
        }
        s_binom[n][k] = c;
    }
    if (threadIdx.x == 0) s_cur = atomicAdd(ep.counter + 1, 1u);
    __syncthreads();

    const V jsum4 = (V)bl.jsum4;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t wic = threadIdx.x >> 5;
    const int Ls = s.L - w.S;
    const int e_lo = bl.n_lo;
    for (;;) {
        const uint32_t blk = s_cur;
        if (blk >= w.nblocks) break;
        if (threadIdx.x == 0) s_next = atomicAdd(ep.counter + 1, 1u);  // next claim, read after the barriers
        const uint32_t h = blk >> w.S, top = blk & ((1u << w.S) - 1u);
        const int c = s.K - __popc(h);          // set bits of the full low pattern
        const int cs = c - __popc(top);         // set bits below the top S bits
        if (c >= 0 && c <= s.L && cs >= 0 && cs <= Ls) {
            const uint32_t rh = __ldg(s.thi + h);
            uint32_t off = 0;
            for (uint32_t t2 = 0; t2 < top; ++t2) {
                const int k2 = c - __popc(t2);
                off += (k2 >= 0 && k2 <= Ls) ? s_binom[Ls][k2] : 0u;
            }
            const uint32_t r0 = rh + off, n = s_binom[Ls][cs];
            // stage the block's rows
            {
                constexpr int RB = B * (int)sizeof(V);
                if constexpr (RB % 16 == 0) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(x + (size_t)r0 * B);
                    uint4 *dst = reinterpret_cast<uint4 *>(s_x);
                    const uint32_t nw = n * (RB / 16);
                    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = __ldg(src + i);
                } else {
                    const V *src = x + (size_t)r0 * B;
                    const uint32_t nw = n * B;
                    for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) s_x[i] = __ldg(src + i);
                }
            }
            __syncthreads();
            const uint32_t uo = __ldg(s.uoff + c);  // start of popcount group c in ulo
            for (uint32_t k0 = wic * 32u; k0 < n; k0 += blockDim.x) {
                const uint32_t k = k0 + lane;
                const bool ok = k < n;
                const uint32_t kk = ok ? k : n - 1;
                const uint32_t r_lo = off + kk;
                const uint32_t l = __ldg(s.ulo + uo + r_lo);
                const uint32_t nl = (h << s.L) | l;
                V acc[B], dsum = (V)0;
#pragma unroll
                for (int r = 0; r < B; ++r) acc[r] = (V)0;
                Chunk<V, C> ch;
                for (int b0 = 0; b0 < bl.nb; b0 += C) {
                    load_chunk(s_bond, b0, ch);
                    bool aa[C];
                    uint32_t src[C];
#pragma unroll
                    for (int q = 0; q < C; ++q) {
                        if (b0 < e_lo) {  // low-low: same group, rank r_hi + tlo
                            const uint32_t m = ch.mlo[q], xm = l & m;
                            aa[q] = (xm != 0u) & (xm != m);
                            src[q] = rh + s_tlo[l ^ m];
                        } else {          // any bond, full label
                            const uint32_t m = ch.mlo[q], xm = nl & m;  // N <= 32: the full mask
                            aa[q] = (xm != 0u) & (xm != m);
                            const uint32_t nn = nl ^ m;
                            src[q] = aa[q] ? __ldg(s.thi + (nn >> s.L)) + s_tlo[nn & s.lomask] : 0u;
                        }
                    }
                    V xv[C][B];
#pragma unroll
                    for (int q = 0; q < C; ++q) {
                        const uint32_t loc = src[q] - r0;
                        if (aa[q] && loc < n) ld_row_smem<B>(s_x + (size_t)loc * B, xv[q]);
                        else if (aa[q]) ld_vec<B>(x + (size_t)src[q] * B, xv[q], false);
                        else {
#pragma unroll
                            for (int r = 0; r < B; ++r) xv[q][r] = (V)0;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < C; ++q)
                        if (aa[q]) {
#pragma unroll
                            for (int r = 0; r < B; ++r) acc[r] = fma(ch.jh[q], xv[q][r], acc[r]);
                            dsum += ch.jh[q];
                        }
                }
                if (ok) {
                    const uint32_t t = r0 + k;
                    V xt[B], up[B], out[B];
                    ld_row_smem<B>(s_x + (size_t)k * B, xt);
                    if (ep.has_prev) ld_vec<B>(y + (size_t)t * B, up, true);
                    const V diag = jsum4 - dsum;
#pragma unroll
                    for (int r = 0; r < B; ++r) {
                        const V hv = fma(diag, xt[r], acc[r]);
                        out[r] = ep.has_prev ? fma(-s_c_prev[r], up[r], hv * s_inv_s[r]) : hv * s_inv_s[r];
                    }
                    st_vec<B>(y + (size_t)t * B, out);
                }
            }
        }
        __syncthreads();  // the block's rows are done; s_next holds the next claim
        if (threadIdx.x == 0) s_cur = s_next;
        __syncthreads();
    }
    if (threadIdx.x == 0) {  // the last CTA to finish zeroes the claim counters
        __threadfence();
        if (atomicAdd(ep.counter + 2, 1u) == gridDim.x - 1) {
            ep.counter[1] = 0;
            ep.counter[2] = 0;
        }
    }
}

template <typename V, int B, int C>
ftlm_status launch_typed(const ftlm_basis *b, const V *x, V *y, const EpiDev &ep, cudaStream_t stream)
{
    const uint64_t row_bytes = (uint64_t)B * sizeof(V);
    StagedWalk w{};
    const int L = b->L;
    for (w.S = 0; w.S <= L; ++w.S) {  // smallest split whose largest block fits
        const int Ls = L - w.S;
        uint64_t c = 1;
        for (int j = 1; j <= Ls / 2; ++j) c = c * (uint64_t)(Ls - Ls / 2 + j) / (uint64_t)j;
        if (c * row_bytes <= kStageBytes) {
            w.cap = (uint32_t)c;
            break;
        }
    }
    if (w.S > L || (b->H << w.S) >= (1ull << 32)) return fail(FTLM_EUNSUPPORTED, "no staged walk for this sector");
    w.nblocks = (uint32_t)(b->H << w.S);
    const size_t smem = (size_t)w.cap * row_bytes + ((size_t)1 << L) * sizeof(uint16_t);
    auto kern = walk_a_staged_kernel<V, B, C>;
    FTLM_CUDA(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 1;
    FTLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStageThreads, smem));
    occ = std::max(1, std::min(occ, 2));
    kern<<<b->num_sms * occ, kStageThreads, smem, stream>>>(b->tables(), b->bonds_walk_a, w, x, y, ep);
    note_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

template <typename V>
ftlm_status launch_width(const ftlm_basis *b, int B, const void *x, void *y, const EpiDev &ep, cudaStream_t stream)
{
    const V *xv = (const V *)x;
    V *yv = (V *)y;
    // bonds per chunk: as many gathers in flight as the 128 registers of two CTAs
    // per SM hold without spilling
    constexpr bool F64 = sizeof(V) == 8;
    switch (B) {
    case 16: return launch_typed<V, 16, F64 ? 1 : 4>(b, xv, yv, ep, stream);
    case 8: return launch_typed<V, 8, F64 ? 2 : 4>(b, xv, yv, ep, stream);
    case 4: return launch_typed<V, 4, F64 ? 4 : 8>(b, xv, yv, ep, stream);
    case 1: return launch_typed<V, 1, 8>(b, xv, yv, ep, stream);
    default: return fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    }
}

}  // namespace

ftlm_status launch_walk_a_staged(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y,
                                 const EpiDev &ep, cudaStream_t stream)
{
    if (b->N > 32 || b->N <= b->L) return fail(FTLM_EUNSUPPORTED, "staged walk needs L < N <= 32");
    return dtype == FTLM_F32 ? launch_width<float>(b, B, x, y, ep, stream)
                             : launch_width<double>(b, B, x, y, ep, stream);
}

}  // namespace ftlm
