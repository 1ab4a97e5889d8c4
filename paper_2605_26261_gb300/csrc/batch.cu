// Batched FTLM chains for many sectors at once (steps a2, a4, a5 over a batch).
//
// A batch lists sectors (of one or many clusters) with R chains each, routed by
// size:
//  - spin-1/2 sectors of dimension above kSmallRows with N <= 32, and every
//    general-spin sector, run the multi-sector path (msv.cu): units of B chains
//    of many sectors advance together, two launches per Lanczos step per wave, on
//    a stream forked from the caller's;
//  - spin-1/2 sectors above kSmallRows with N > 32 run the grid-wide launch
//    sequence of ftlm_lanczos on up to kMaxSideStreams side streams (longest work
//    first, each to the least-loaded stream);
//  - all smaller sectors are cut into work units of B chains and handed to ONE
//    persistent launch on the caller's stream: each CTA takes the next unit
// from an atomic counter (no waiting on other CTAs) and runs the unit's whole
// chains by itself -- start vectors, min(M, D) steps of fused H.v + Lanczos
// update with CTA-local reductions, stop tests -- with the unit's two vector blocks
// in a per-CTA slot of the workspace (L2-resident for small sectors).  One Ritz
// launch then handles every chain of the small sectors, and a scatter copies the
// results into each sector's outputs.  Units are sorted by dimension, largest
// first, so the tail of the queue is short work.
//
// The plan (descriptors of sectors and units) is uploaded once by
// ftlm_batch_create; ftlm_batch_run only issues memsets and kernel launches, so the
// whole run can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ftlm_internal.cuh"
#include "msv.cuh"
#include "reduce.cuh"
#include "rng.cuh"
#include "rows.cuh"
#include "vec.cuh"

namespace ftlm {

// Vector bytes of one wave of the multi-sector path: FTLM_MS_WAVE_MB or 256 MB.
// Small waves keep a wave's vectors near the L2 size (measured on GB300 with 256
// clusters of 18-22 sites: 256 MB waves 9.6 s per run, 2 GB 11.0 s, 8 GB 11.9 s);
// a unit larger than the budget forms a wave of its own.
uint64_t ms_wave_bytes()
{
    static const uint64_t v = [] {
        const char *e = std::getenv("FTLM_MS_WAVE_MB");
        const long long mb = e ? std::atoll(e) : 256;
        return (uint64_t)(mb > 0 ? mb : 256) << 20;
    }();
    return v;
}

namespace {

constexpr int kBatchThreads = 256;
constexpr uint64_t kSmallRows = 1u << 15;  // sectors up to this dimension run inside one CTA
constexpr int kMaxSideStreams = 8;


// Default number of side streams for the large items: FTLM_BATCH_STREAMS (1..8)
// or 4.
int side_streams()
{
    static const int n = [] {
        const char *v = std::getenv("FTLM_BATCH_STREAMS");
        const int k = v ? std::atoi(v) : 4;
        return std::max(1, std::min(kMaxSideStreams, k));
    }();
    return n;
}

struct BatchItemDev {
    SectorTables s;
    BondList bl;
    uint64_t seed;
    double tau;
    int chain0;  // key index of the item's first chain
    int m_max;
    int N, K;
    uint32_t chain_base;  // index of the item's chain 0 among the batch's small chains
    int pad;
};

struct BatchUnitDev {
    uint32_t item;  // index into the item descriptors
    uint32_t r0;    // first chain of the unit within the item
    uint32_t nact;  // chains of the unit (<= B); the other columns stay zero
    uint32_t pad;
};

struct ScatterDev {
    double *theta;  // row of the chain in the item's outputs
    double *weight;
    int *m_eff;
};

// Fixed-order CTA sum of B per-thread accumulators (one transposed warp tree, then
// the warp sums in warp order); out[r] (shared) holds chain r's total.
template <typename V, int B>
__device__ __forceinline__ void cta_reduce(DotAcc<V> (&v)[B], double *s_warp, double *out)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const DotAcc<V> t = warp_sum_multi<V, B>(v);
    if (lane < B) s_warp[w * B + warp_multi_index<B>(lane)] = t.value();
    __syncthreads();
    if (threadIdx.x < B) {
        double t = 0.0;
        for (int i = 0; i < kBatchThreads / 32; ++i) t += s_warp[i * B + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

template <typename V, typename Lbl, bool CLT, int B, int C>
__global__ void __launch_bounds__(kBatchThreads)
batch_kernel(const BatchItemDev *__restrict__ items, const BatchUnitDev *__restrict__ units, uint32_t n_units,
             unsigned int *queue, V *slots, uint64_t slot_elems, int M, int dist, double *alpha_all,
             double *beta_all, int *meff_all)
{
    extern __shared__ uint16_t s_tlo[];
    __shared__ uint4 s_bond[kMaxBondSlots];
    __shared__ double s_warp[(kBatchThreads / 32) * B];
    __shared__ double s_tot[B], s_cur[B], s_prev[B], s_bprev[B];
    __shared__ V s_inv_s[B], s_cprev[B], s_a[B];
    __shared__ int s_stop[B], s_meff[B];
    __shared__ unsigned int s_unit;
    __shared__ int s_all_stopped;
    V *const u0 = slots + (size_t)blockIdx.x * 2 * slot_elems;
    V *const u1 = u0 + slot_elems;

    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(queue, 1u);
        __syncthreads();
        const unsigned int ui = s_unit;
        if (ui >= n_units) break;  // CTA-uniform
        const BatchUnitDev un = units[ui];
        const SectorTables s = items[un.item].s;
        const BondList bl = items[un.item].bl;
        const BatchItemDev &it = items[un.item];
        const uint32_t D = s.D;
        const int m_max = it.m_max;
        const double tau = it.tau;
        const size_t cbase = (size_t)it.chain_base + un.r0;
        {
            const uint4 *src = sizeof(V) == 4 ? bl.slots_f32 : bl.slots_f64;
            for (int i = threadIdx.x; i < bl.nb; i += kBatchThreads) s_bond[i] = src[i];
            if (!CLT)
                for (uint32_t i = threadIdx.x; i <= s.lomask; i += kBatchThreads) s_tlo[i] = __ldg(s.tlo + i);
        }
        // start vectors of the unit's chains (columns past nact stay zero)
        {
            uint64_t key[B];
#pragma unroll
            for (int r = 0; r < B; ++r) key[r] = chain_key(it.seed, it.N, it.K, (uint32_t)(it.chain0 + un.r0 + r));
            DotAcc<V> acc[B];
            for (uint32_t t = threadIdx.x; t < D; t += kBatchThreads) {
                V out[B];
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    out[r] = r < (int)un.nact ? (V)start_value(key[r], t, dist) : (V)0;
                    acc[r].add(out[r], out[r]);
                }
                st_vec<B>(u0 + (size_t)t * B, out);
            }
            cta_reduce<V, B>(acc, s_warp, s_tot);
            if (threadIdx.x < B) {
                const int r = threadIdx.x;
                const double nrm = sqrt(s_tot[r]);
                s_cur[r] = nrm;
                s_prev[r] = 1.0;
                s_bprev[r] = 0.0;
                s_stop[r] = (r < (int)un.nact && nrm > 0.0 && isfinite(nrm)) ? 0 : 1;
                s_meff[r] = 0;
            }
            __syncthreads();
        }
        int cur = 0;
        for (int j = 1; j <= m_max; ++j) {
            if (threadIdx.x < B) {
                const int r = threadIdx.x;
                s_inv_s[r] = (V)(1.0 / s_cur[r]);
                s_cprev[r] = j > 1 ? (V)(s_bprev[r] / s_prev[r]) : (V)0;
            }
            if (threadIdx.x == 0) {
                int all = 1;
                for (int r = 0; r < B; ++r) all &= s_stop[r];
                s_all_stopped = all;
            }
            __syncthreads();
            if (s_all_stopped) break;  // CTA-uniform
            const V *x = cur ? u1 : u0;
            V *y = cur ? u0 : u1;
            // y = H q_j - beta_{j-1} q_{j-1} (over u_{j-1}), alpha partials
            DotAcc<V> ap[B];
            for (uint32_t t = threadIdx.x; t < D; t += kBatchThreads) {
                const uint32_t tt[1] = {t};
                V acc[1][B], dsum[1] = {(V)0};
#pragma unroll
                for (int r = 0; r < B; ++r) acc[0][r] = (V)0;
                if (CLT) rows_clt<V, 1, B, C, false>(s, bl, s_bond, x, tt, acc, dsum);
                else rows_cr<V, Lbl, 1, B, C, false>(s, bl, s_bond, s_tlo, x, tt, acc, dsum);
                V xt[B], up[B], out[B];
                ld_vec_coherent<B>(x + (size_t)t * B, xt);
                if (j > 1) ld_vec_coherent<B>(y + (size_t)t * B, up);
                const V diag = (V)bl.jsum4 - dsum[0];
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const V hv = fma(diag, xt[r], acc[0][r]);
                    out[r] = j > 1 ? fma(-s_cprev[r], up[r], hv * s_inv_s[r]) : hv * s_inv_s[r];
                    ap[r].add(xt[r] * s_inv_s[r], out[r]);
                }
                st_vec<B>(y + (size_t)t * B, out);
            }
            cta_reduce<V, B>(ap, s_warp, s_tot);
            if (threadIdx.x < B) {
                const int r = threadIdx.x;
                if (!s_stop[r]) alpha_all[(cbase + r) * M + (j - 1)] = s_tot[r];
                s_a[r] = s_stop[r] ? (V)0 : (V)(s_tot[r] / s_cur[r]);
            }
            __syncthreads();
            // w = y - alpha_j q_j in place, beta_j = ||w||
            DotAcc<V> bp[B];
            for (uint32_t t = threadIdx.x; t < D; t += kBatchThreads) {
                V yv[B], xv[B], w[B];
                ld_vec_coherent<B>(y + (size_t)t * B, yv);
                ld_vec_coherent<B>(x + (size_t)t * B, xv);
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    w[r] = s_stop[r] ? (V)0 : fma(-s_a[r], xv[r], yv[r]);
                    bp[r].add(w[r], w[r]);
                }
                st_vec<B>(y + (size_t)t * B, w);
            }
            cta_reduce<V, B>(bp, s_warp, s_tot);
            if (threadIdx.x < B && !s_stop[threadIdx.x]) {
                const int r = threadIdx.x;
                const double beta = sqrt(s_tot[r]);
                if (j < m_max) {
                    if (beta <= tau) {
                        s_stop[r] = 1;
                        s_meff[r] = j;
                    } else {
                        beta_all[(cbase + r) * M + (j - 1)] = beta;
                        s_prev[r] = s_cur[r];
                        s_cur[r] = beta;
                        s_bprev[r] = beta;
                    }
                } else {
                    s_meff[r] = m_max;
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        if (threadIdx.x < un.nact) meff_all[cbase + threadIdx.x] = s_meff[threadIdx.x];
        __syncthreads();  // the next unit reuses shared memory and the slot
    }
}

__global__ void scatter_kernel(int n, int M, const double *__restrict__ theta, const double *__restrict__ weight,
                               const int *__restrict__ meff, const ScatterDev *__restrict__ dst)
{
    const int c = blockIdx.x;
    if (c >= n) return;
    const ScatterDev d = dst[c];
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        d.theta[k] = theta[(size_t)c * M + k];
        d.weight[k] = weight[(size_t)c * M + k];
    }
    if (threadIdx.x == 0) *d.m_eff = meff[c];
}

uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

// Kernel variant of a group of units: rank mode and label width.
enum Group { kCr32 = 0, kCr64 = 1, kClt = 2 };

template <typename V, int B>
void *batch_kernel_ptr(int group)
{
    constexpr int C = B >= 8 ? 4 : kBondChunk;
    if (group == kClt) return (void *)batch_kernel<V, uint32_t, true, B, C>;
    if (group == kCr64) return (void *)batch_kernel<V, uint64_t, false, B, C>;
    return (void *)batch_kernel<V, uint32_t, false, B, C>;
}

void *kernel_for(ftlm_dtype dtype, int B, int group)
{
    if (dtype == FTLM_F32) {
        switch (B) {
        case 16: return batch_kernel_ptr<float, 16>(group);
        case 8: return batch_kernel_ptr<float, 8>(group);
        case 4: return batch_kernel_ptr<float, 4>(group);
        default: return batch_kernel_ptr<float, 1>(group);
        }
    }
    switch (B) {
    case 16: return batch_kernel_ptr<double, 16>(group);
    case 8: return batch_kernel_ptr<double, 8>(group);
    case 4: return batch_kernel_ptr<double, 4>(group);
    default: return batch_kernel_ptr<double, 1>(group);
    }
}

}  // namespace

}  // namespace ftlm

using namespace ftlm;

struct ftlm_batch {
    int n, M, dist, B;
    ftlm_dtype dtype;
    std::vector<ftlm_batch_item> items;
    std::vector<int> large;     // items run through the launch sequence of ftlm_lanczos
    uint32_t n_small_chains;
    uint32_t n_chains;          // small chains, then the chains of the multi-sector path
    uint32_t group_units[3];    // units per kernel variant
    uint32_t group_first[3];    // offset of the group in the unit array
    int group_grid[3];
    int n_slots;
    uint64_t slot_elems;        // D_max * B of the small items
    // device descriptors (owned): one pooled block holding the three arrays
    void *desc_block;
    BatchItemDev *d_items;
    BatchUnitDev *d_units;
    ScatterDev *d_scatter;
    // workspace layout
    uint64_t off_queue, off_slots, off_alpha, off_beta, off_meff, off_theta, off_weight, off_large, total;
    uint64_t large_bytes;       // workspace of one large item (the largest)
    // large items run on side streams forked from the caller's stream, each with
    // its own workspace region; large_side[k] is the side stream of large[k]
    int n_side;
    cudaStream_t side[kMaxSideStreams];
    cudaEvent_t ev_fork, ev_join[kMaxSideStreams];
    std::vector<int> large_side;
    // multi-sector path (msv.cu): units of B chains of the mid-sized and large
    // spin-1/2 sectors, run in waves on their own stream
    std::vector<MsWave> waves;
    MsUnit *d_ms_units;
    uint32_t *d_tile_unit;
    uint32_t *d_stile_unit;
    uint64_t off_ms;
    int num_sms;
    cudaStream_t ms_stream;
    cudaEvent_t ev_ms_join;
};

namespace {

void release_host_objects(ftlm_batch *p)
{
    for (int k = 0; k < p->n_side; ++k) {
        if (p->side[k]) cudaStreamDestroy(p->side[k]);
        if (p->ev_join[k]) cudaEventDestroy(p->ev_join[k]);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ms_stream) cudaStreamDestroy(p->ms_stream);
    if (p->ev_ms_join) cudaEventDestroy(p->ev_ms_join);
    delete p;
}

}  // namespace

namespace {

ftlm_status batch_create(int n, const ftlm_batch_item *items, int M, ftlm_vec_dist dist, ftlm_dtype dtype, int block,
                         int streams, uint32_t tile_rows, uint32_t stream_rows, void *stream_, ftlm_batch **out)
{
    if (!out) return fail(FTLM_EINVAL, "out is NULL");
    if (tile_rows == 0) tile_rows = kMsTileRows;
    if (stream_rows == 0) stream_rows = kMsStreamRows;
    if (tile_rows % kRowThreads || stream_rows % kRowThreads || tile_rows > (1u << 20) || stream_rows > (1u << 20))
        return fail(FTLM_EINVAL, "tile rows must be multiples of 256 up to 2^20");
    *out = nullptr;
    if (n < 1 || !items) return fail(FTLM_EINVAL, "empty batch");
    if (M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "M out of range");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    if (dist != FTLM_VEC_GAUSS && dist != FTLM_VEC_RADEMACHER) return fail(FTLM_EINVAL, "bad distribution");
    if (block == 0) block = dtype == FTLM_F32 ? 16 : 8;
    if (!valid_block(block)) return fail(FTLM_EINVAL, "block width must be 0, 1, 4, 8 or 16");
    if (streams < 0 || streams > kMaxSideStreams) return fail(FTLM_EINVAL, "streams must be 0..8");
    if (streams == 0) streams = side_streams();
    for (int i = 0; i < n; ++i) {
        const ftlm_batch_item &it = items[i];
        if (!it.basis || it.R < 1 || it.first_chain < 0) return fail(FTLM_EINVAL, "bad batch item");
        if (!it.theta_dev || !it.weight_dev || !it.m_eff_dev) return fail(FTLM_EINVAL, "NULL output in batch item");
    }
    ftlm_batch *p = new (std::nothrow) ftlm_batch();
    if (!p) return fail(FTLM_ENOMEM, "host allocation failed");
    p->n = n;
    p->M = M;
    p->dist = dist;
    p->B = block;
    p->dtype = dtype;
    p->items.assign(items, items + n);
    const int B = block;

    std::vector<BatchItemDev> hitems;
    std::vector<std::vector<BatchUnitDev>> gunits(3);
    std::vector<ScatterDev> scatter;
    std::vector<uint64_t> unit_dim[3];
    uint64_t dmax = 1, large_bytes = 0;
    int num_sms = 0;
    std::vector<int> ms_items;
    for (int i = 0; i < n; ++i) {
        const ftlm_basis *b = items[i].basis;
        num_sms = b->num_sms;
        if (b->two_s > 1 || (b->N <= 32 && b->D > kSmallRows)) {  // the multi-sector path
            ms_items.push_back(i);
            continue;
        }
        if (b->D > kSmallRows) {  // N > 32: the launch sequence of ftlm_lanczos
            p->large.push_back(i);
            large_bytes = std::max<uint64_t>(large_bytes, lanczos_workspace(b, items[i].R, M, dtype, B));
            continue;
        }
        BatchItemDev d{};
        d.s = b->tables();
        d.bl = b->mode == FTLM_RANK_CLT ? b->bonds_clt : b->bonds_cr;
        d.seed = items[i].seed;
        d.tau = dtype == FTLM_F32 ? b->tau32 : b->tau64;
        d.chain0 = items[i].first_chain;
        d.m_max = (uint64_t)M < b->D ? M : (int)b->D;
        d.N = b->N;
        d.K = b->K;
        d.chain_base = p->n_small_chains;
        const int group = b->mode == FTLM_RANK_CLT ? kClt : (b->N > 32 ? kCr64 : kCr32);
        for (int r0 = 0; r0 < items[i].R; r0 += B) {
            BatchUnitDev u{};
            u.item = (uint32_t)hitems.size();
            u.r0 = (uint32_t)r0;
            u.nact = (uint32_t)std::min(B, items[i].R - r0);
            gunits[group].push_back(u);
        }
        for (int r = 0; r < items[i].R; ++r)
            scatter.push_back({items[i].theta_dev + (size_t)r * M, items[i].weight_dev + (size_t)r * M,
                               items[i].m_eff_dev + r});
        p->n_small_chains += (uint32_t)items[i].R;
        dmax = std::max<uint64_t>(dmax, b->D);
        hitems.push_back(d);
    }
    // largest sectors first within each group (the queue's tail is short work)
    std::vector<BatchUnitDev> units;
    for (int g = 0; g < 3; ++g) {
        std::stable_sort(gunits[g].begin(), gunits[g].end(), [&](const BatchUnitDev &a, const BatchUnitDev &b) {
            return hitems[a.item].s.D > hitems[b.item].s.D;
        });
        p->group_first[g] = (uint32_t)units.size();
        p->group_units[g] = (uint32_t)gunits[g].size();
        units.insert(units.end(), gunits[g].begin(), gunits[g].end());
    }
    // persistent grids: resident CTAs of each variant
    p->n_slots = 1;
    const size_t smem = ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
    for (int g = 0; g < 3; ++g) {
        p->group_grid[g] = 0;
        if (!p->group_units[g]) continue;
        void *kern = kernel_for(dtype, B, g);
        int occ = 1;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatchThreads, smem);
        if (e != cudaSuccess) {
            delete p;
            return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)");
        }
        occ = std::max(1, occ);
        p->group_grid[g] = (int)std::min<uint64_t>(p->group_units[g], (uint64_t)num_sms * occ);
        p->n_slots = std::max(p->n_slots, p->group_grid[g]);
    }
    // Multi-sector path: units of B chains, grouped by rank kind, cut into waves of
    // at most ms_wave_bytes() of vectors; offsets within a wave are relative to the
    // ms region of the workspace (each wave reuses it).
    const uint64_t vsize = dtype == FTLM_F32 ? 4 : 8;
    std::vector<MsUnit> ms_units;
    std::vector<uint32_t> tile_unit, stile_unit;
    uint64_t ms_bytes = 0;
    p->n_chains = p->n_small_chains;
    auto kind_of = [](const ftlm_basis *b) {
        return b->two_s > 1 ? kMsSpin : (b->mode == FTLM_RANK_CLT ? kMsClt : kMsCr);
    };
    for (int kind = 0; kind < 3; ++kind) {
        MsWave w{};
        uint64_t wbytes = 0;
        auto close_wave = [&]() {
            if (!w.n_units) return;
            p->waves.push_back(w);
            ms_bytes = std::max(ms_bytes, wbytes);
            w = MsWave{};
            wbytes = 0;
        };
        for (int i : ms_items) {
            const ftlm_basis *b = items[i].basis;
            if (kind_of(b) != kind) continue;
            for (int r0 = 0; r0 < items[i].R; r0 += B) {
                const uint64_t vb = align256(b->D * (uint64_t)B * vsize);
                const uint32_t nt = (uint32_t)((b->D + tile_rows - 1) / tile_rows);
                const uint64_t ub = 2 * vb + align256(kMaxBlock * sizeof(ChainState) + 64) +
                                    align256((uint64_t)nt * B * sizeof(double));
                if (w.n_units && wbytes + ub > ms_wave_bytes()) close_wave();
                if (!w.n_units) {
                    w.unit0 = (uint32_t)ms_units.size();
                    w.tile_off = (uint32_t)tile_unit.size();
                    w.stile_off = (uint32_t)stile_unit.size();
                    w.kind = kind;
                }
                const uint32_t nst = (uint32_t)((b->D + stream_rows - 1) / stream_rows);
                MsUnit u{};
                u.s = b->tables();
                u.bl = b->mode == FTLM_RANK_CLT ? b->bonds_clt : b->bonds_cr;
                u.spin = b->spin;
                u.off_v0 = wbytes;
                u.off_v1 = wbytes + vb;
                u.off_st = wbytes + 2 * vb;
                u.off_part = u.off_st + align256(kMaxBlock * sizeof(ChainState) + 64);
                u.seed = items[i].seed;
                u.tau = dtype == FTLM_F32 ? b->tau32 : b->tau64;
                u.tile_rows = tile_rows;
                u.stream_rows = stream_rows;
                u.tile0 = w.n_tiles;
                u.n_tiles = nt;
                u.stile0 = w.n_stiles;
                u.n_stiles = nst;
                u.chain_base = p->n_chains + (uint32_t)r0;
                u.key_n = b->key_n;
                u.K = b->K;
                u.chain0 = items[i].first_chain + r0;
                u.nact = std::min(B, items[i].R - r0);
                u.m_max = (uint64_t)M < b->D ? M : (int)b->D;
                for (uint32_t k = 0; k < nt; ++k) tile_unit.push_back(w.n_units);  // wave-local unit index
                for (uint32_t k = 0; k < nst; ++k) stile_unit.push_back(w.n_units);
                w.n_units += 1;
                w.n_tiles += nt;
                w.n_stiles += nst;
                w.m_max = std::max(w.m_max, u.m_max);
                wbytes += ub;
                ms_units.push_back(u);
            }
            for (int r = 0; r < items[i].R; ++r)
                scatter.push_back({items[i].theta_dev + (size_t)r * M, items[i].weight_dev + (size_t)r * M,
                                   items[i].m_eff_dev + r});
            p->n_chains += (uint32_t)items[i].R;
        }
        close_wave();
    }
    p->num_sms = num_sms;

    // workspace layout
    p->slot_elems = dmax * (uint64_t)B;
    uint64_t off = 0;
    p->off_queue = off;
    off += 256;
    p->off_slots = off;
    off += align256((uint64_t)p->n_slots * 2 * p->slot_elems * vsize);
    const uint64_t cm = (uint64_t)p->n_chains * M * sizeof(double);
    p->off_alpha = off;
    off += align256(cm);
    p->off_beta = off;
    off += align256(cm);
    p->off_theta = off;
    off += align256(cm);
    p->off_weight = off;
    off += align256(cm);
    p->off_meff = off;
    off += align256((uint64_t)p->n_chains * sizeof(int));
    p->off_ms = off;
    off += ms_bytes;
    // Large items: longest-processing-time assignment to the side streams (the
    // work of a sector's chains grows with D), so they overlap one another and the
    // persistent kernel of the small items.
    p->n_side = (int)std::min<size_t>(p->large.size(), (size_t)streams);
    if (p->n_side) {
        std::vector<int> order(p->large.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return items[p->large[a]].basis->D * (uint64_t)items[p->large[a]].R >
                   items[p->large[b]].basis->D * (uint64_t)items[p->large[b]].R;
        });
        std::vector<uint64_t> load(p->n_side, 0);
        p->large_side.assign(p->large.size(), 0);
        for (int k : order) {
            const int sidx = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            p->large_side[k] = sidx;
            load[sidx] += items[p->large[k]].basis->D * (uint64_t)items[p->large[k]].R;
        }
    }
    large_bytes = align256(large_bytes);
    p->off_large = off;
    off += large_bytes * (uint64_t)std::max(1, p->n_side);
    p->large_bytes = large_bytes;
    p->total = off;

    // descriptors to the device: one pooled block, one copy
    cudaStream_t stream = (cudaStream_t)stream_;
    const uint64_t o_items = 0;
    const uint64_t o_units = align256(o_items + hitems.size() * sizeof(BatchItemDev));
    const uint64_t o_scatter = align256(o_units + units.size() * sizeof(BatchUnitDev));
    const uint64_t o_ms = align256(o_scatter + scatter.size() * sizeof(ScatterDev));
    const uint64_t o_tiles = align256(o_ms + ms_units.size() * sizeof(MsUnit));
    const uint64_t o_stiles = align256(o_tiles + tile_unit.size() * sizeof(uint32_t));
    const uint64_t desc_bytes = std::max<uint64_t>(256, align256(o_stiles + stile_unit.size() * sizeof(uint32_t)));
    std::vector<unsigned char> image(desc_bytes, 0);
    if (!hitems.empty()) std::memcpy(image.data() + o_items, hitems.data(), hitems.size() * sizeof(BatchItemDev));
    if (!units.empty()) std::memcpy(image.data() + o_units, units.data(), units.size() * sizeof(BatchUnitDev));
    if (!scatter.empty())
        std::memcpy(image.data() + o_scatter, scatter.data(), scatter.size() * sizeof(ScatterDev));
    if (!ms_units.empty()) std::memcpy(image.data() + o_ms, ms_units.data(), ms_units.size() * sizeof(MsUnit));
    if (!tile_unit.empty())
        std::memcpy(image.data() + o_tiles, tile_unit.data(), tile_unit.size() * sizeof(uint32_t));
    if (!stile_unit.empty())
        std::memcpy(image.data() + o_stiles, stile_unit.data(), stile_unit.size() * sizeof(uint32_t));
    int device = 0;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = table_pool(device, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&p->desc_block, desc_bytes, pool, stream);
    if (e == cudaSuccess) {
        char *base = static_cast<char *>(p->desc_block);
        p->d_items = reinterpret_cast<BatchItemDev *>(base + o_items);
        p->d_units = reinterpret_cast<BatchUnitDev *>(base + o_units);
        p->d_scatter = reinterpret_cast<ScatterDev *>(base + o_scatter);
        p->d_ms_units = reinterpret_cast<MsUnit *>(base + o_ms);
        p->d_tile_unit = reinterpret_cast<uint32_t *>(base + o_tiles);
        p->d_stile_unit = reinterpret_cast<uint32_t *>(base + o_stiles);
        e = cudaMemcpyAsync(base, image.data(), desc_bytes, cudaMemcpyHostToDevice, stream);
    }
    for (int g = 0; g < 3 && e == cudaSuccess; ++g)
        if (p->group_units[g])
            e = cudaFuncSetAttribute(kernel_for(dtype, B, g), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && (p->n_side || !p->waves.empty()))
        e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !p->waves.empty()) {
        e = cudaStreamCreateWithFlags(&p->ms_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_ms_join, cudaEventDisableTiming);
    }
    for (int k = 0; k < p->n_side && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&p->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        if (p->desc_block) cudaFreeAsync(p->desc_block, stream);
        release_host_objects(p);
        return e == cudaErrorMemoryAllocation ? fail(FTLM_ENOMEM, "no device memory for the batch descriptors")
                                              : cuda_fail(e, "batch descriptors");
    }
    *out = p;
    return FTLM_OK;
}

}  // namespace

extern "C" ftlm_status ftlm_batch_create(int n, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                         ftlm_dtype dtype, int block, int streams, void *stream, ftlm_batch **out)
{
    return batch_create(n, items, M, dist, dtype, block, streams, 0, 0, stream, out);
}

extern "C" ftlm_status ftlm_batch_create_plan(int n, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                              ftlm_dtype dtype, const ftlm_batch_plan *plan, void *stream,
                                              ftlm_batch **out)
{
    if (!plan) return fail(FTLM_EINVAL, "NULL plan");
    if (plan->tile_rows < 0 || plan->stream_rows < 0) return fail(FTLM_EINVAL, "negative tile rows");
    return batch_create(n, items, M, dist, dtype, plan->block, plan->streams, (uint32_t)plan->tile_rows,
                        (uint32_t)plan->stream_rows, stream, out);
}

extern "C" void ftlm_batch_destroy(ftlm_batch *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFreeAsync(p->desc_block, 0);
    release_host_objects(p);
}

extern "C" ftlm_status ftlm_batch_destroy_async(ftlm_batch *p, void *stream)
{
    if (!p) return FTLM_OK;
    const cudaError_t e = cudaFreeAsync(p->desc_block, (cudaStream_t)stream);
    release_host_objects(p);  // stream and event destruction waits for their work
    return e == cudaSuccess ? FTLM_OK : cuda_fail(e, "cudaFreeAsync(batch descriptors)");
}

extern "C" ftlm_status ftlm_batch_workspace_bytes(const ftlm_batch *p, uint64_t *bytes)
{
    if (!p || !bytes) return fail(FTLM_EINVAL, "NULL argument");
    *bytes = p->total;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_batch_run(const ftlm_batch *p, void *work_dev, uint64_t work_bytes, void *stream_)
{
    if (!p) return fail(FTLM_EINVAL, "NULL batch");
    if (!work_dev || ((uintptr_t)work_dev & 255u)) return fail(FTLM_EINVAL, "workspace NULL or not 256-byte aligned");
    if (work_bytes < p->total) return fail(FTLM_ENOMEM, "workspace smaller than ftlm_batch_workspace_bytes()");
    cudaStream_t stream = (cudaStream_t)stream_;
    char *ws = (char *)work_dev;
    const int M = p->M;
    unsigned int *queues = (unsigned int *)(ws + p->off_queue);
    double *alpha = (double *)(ws + p->off_alpha), *beta = (double *)(ws + p->off_beta);
    double *theta = (double *)(ws + p->off_theta), *weight = (double *)(ws + p->off_weight);
    int *meff = (int *)(ws + p->off_meff);
    if (p->n_chains) {
        const size_t cm = (size_t)p->n_chains * M * sizeof(double);
        FTLM_CUDA(cudaMemsetAsync(queues, 0, 3 * sizeof(unsigned int), stream));
        FTLM_CUDA(cudaMemsetAsync(alpha, 0, cm, stream));
        FTLM_CUDA(cudaMemsetAsync(beta, 0, cm, stream));
    }
    if (p->n_side || !p->waves.empty()) FTLM_CUDA(cudaEventRecord(p->ev_fork, stream));
    // multi-sector path on its own stream, overlapping the persistent kernel
    if (!p->waves.empty()) {
        FTLM_CUDA(cudaStreamWaitEvent(p->ms_stream, p->ev_fork, 0));
        for (const MsWave &w : p->waves) {
            ftlm_status s = ms_run_wave(w, p->dtype, p->B, p->d_ms_units + w.unit0, p->d_tile_unit + w.tile_off,
                                        p->d_stile_unit + w.stile_off, M, p->dist, ws + p->off_ms, alpha, beta, meff,
                                        p->num_sms, p->ms_stream);
            if (s != FTLM_OK) return s;
        }
        FTLM_CUDA(cudaEventRecord(p->ev_ms_join, p->ms_stream));
    }
    // general-spin and N > 32 sectors on the side streams
    if (p->n_side) {
        for (int k = 0; k < p->n_side; ++k) FTLM_CUDA(cudaStreamWaitEvent(p->side[k], p->ev_fork, 0));
        for (size_t k = 0; k < p->large.size(); ++k) {
            const ftlm_batch_item &it = p->items[p->large[k]];
            const int sidx = p->large_side[k];
            ftlm_status s = lanczos_run(it.basis, it.R, M, it.first_chain, it.seed, p->dist, nullptr, p->dtype,
                                        ws + p->off_large + (uint64_t)sidx * p->large_bytes, p->large_bytes,
                                        it.theta_dev, it.weight_dev, it.m_eff_dev, nullptr, nullptr, p->side[sidx],
                                        p->B);
            if (s != FTLM_OK) return s;
        }
    }
    // small sectors: one persistent launch per kernel variant
    if (p->n_small_chains) {
        const size_t smem = ((size_t)1 << kLoBitsMax) * sizeof(uint16_t);
        for (int g = 0; g < 3; ++g) {
            if (!p->group_units[g]) continue;
            void *kern = kernel_for(p->dtype, p->B, g);
            const BatchItemDev *items = p->d_items;
            const BatchUnitDev *units = p->d_units + p->group_first[g];
            uint32_t n_units = p->group_units[g];
            unsigned int *queue = queues + g;
            void *slots = ws + p->off_slots;
            uint64_t slot_elems = p->slot_elems;
            int Mi = M, dist = p->dist;
            void *args[] = {(void *)&items, (void *)&units, (void *)&n_units, (void *)&queue, (void *)&slots,
                            (void *)&slot_elems, (void *)&Mi, (void *)&dist, (void *)&alpha, (void *)&beta,
                            (void *)&meff};
            FTLM_CUDA(cudaLaunchKernel(kern, dim3(p->group_grid[g]), dim3(kBatchThreads), args, smem, stream));
            note_launch();
        }
    }
    // Ritz step of every chain of both paths, results to the items' outputs
    if (!p->waves.empty()) FTLM_CUDA(cudaStreamWaitEvent(stream, p->ev_ms_join, 0));
    if (p->n_chains) {
        ftlm_status s = launch_ritz((int)p->n_chains, M, alpha, beta, meff, theta, weight, stream);
        if (s != FTLM_OK) return s;
        scatter_kernel<<<p->n_chains, 128, 0, stream>>>((int)p->n_chains, M, theta, weight, meff, p->d_scatter);
        note_launch();
        FTLM_CUDA(cudaGetLastError());
    }
    for (int k = 0; k < p->n_side; ++k) {
        FTLM_CUDA(cudaEventRecord(p->ev_join[k], p->side[k]));
        FTLM_CUDA(cudaStreamWaitEvent(stream, p->ev_join[k], 0));
    }
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_batch_autotune(int n, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                           ftlm_dtype dtype, void *stream_, int *block_out, int *streams_out,
                                           float *ms_out)
{
    if (!block_out || !streams_out) return fail(FTLM_EINVAL, "NULL output");
    cudaStream_t stream = (cudaStream_t)stream_;
    // the stream count matters only for items on the side streams (general spin, N > 32)
    bool any_large = false;
    for (int i = 0; i < n && items; ++i) {
        const ftlm_basis *b = items[i].basis;
        if (b && b->two_s == 1 && b->N > 32 && b->D > kSmallRows) any_large = true;
    }
    int device = 0;
    cudaMemPool_t pool = nullptr;
    FTLM_CUDA(cudaGetDevice(&device));
    FTLM_CUDA(table_pool(device, &pool));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    FTLM_CUDA(cudaEventCreate(&ev[0]));
    FTLM_CUDA(cudaEventCreate(&ev[1]));
    float best = -1.f;
    int best_b = 0, best_s = 0;
    ftlm_status st = FTLM_OK;
    const int blocks[3] = {4, 8, 16};
    const int streams_try[4] = {1, 2, 4, 8};
    for (int bi = 0; bi < 3 && st == FTLM_OK; ++bi) {
        for (int si = 0; si < (any_large ? 4 : 1) && st == FTLM_OK; ++si) {
            ftlm_batch *p = nullptr;
            st = ftlm_batch_create(n, items, M, dist, dtype, blocks[bi], streams_try[si], stream, &p);
            if (st != FTLM_OK) break;
            void *work = nullptr;
            cudaError_t e = cudaMallocFromPoolAsync(&work, p->total, pool, stream);
            if (e != cudaSuccess) {
                ftlm_batch_destroy_async(p, stream);
                st = e == cudaErrorMemoryAllocation ? fail(FTLM_ENOMEM, "no device memory for a tuning run")
                                                    : cuda_fail(e, "cudaMallocFromPoolAsync(tuning workspace)");
                break;
            }
            // one untimed run, then one timed run
            st = ftlm_batch_run(p, work, p->total, stream);
            if (st == FTLM_OK && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) st = cuda_fail(e, "event");
            if (st == FTLM_OK) st = ftlm_batch_run(p, work, p->total, stream);
            if (st == FTLM_OK && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) st = cuda_fail(e, "event");
            if (st == FTLM_OK && (e = cudaEventSynchronize(ev[1])) != cudaSuccess) st = cuda_fail(e, "tuning run");
            float ms = 0.f;
            if (st == FTLM_OK && (e = cudaEventElapsedTime(&ms, ev[0], ev[1])) != cudaSuccess)
                st = cuda_fail(e, "cudaEventElapsedTime");
            cudaFreeAsync(work, stream);
            ftlm_batch_destroy_async(p, stream);
            if (st != FTLM_OK) break;
            if (ms_out) ms_out[bi * 4 + si] = ms;
            if (best < 0.f || ms < best) {
                best = ms;
                best_b = blocks[bi];
                best_s = streams_try[si];
            }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != FTLM_OK) return st;
    *block_out = best_b;
    *streams_out = best_s;
    return FTLM_OK;
}

namespace {

// One timed run of a plan (after one untimed run); ms in *ms.
ftlm_status time_plan(int n, const ftlm_batch_item *items, int M, ftlm_vec_dist dist, ftlm_dtype dtype,
                      const ftlm_batch_plan &pl, cudaStream_t stream, cudaMemPool_t pool, cudaEvent_t *ev, float *ms)
{
    ftlm_batch *p = nullptr;
    ftlm_status st = ftlm_batch_create_plan(n, items, M, dist, dtype, &pl, stream, &p);
    if (st != FTLM_OK) return st;
    void *work = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&work, p->total, pool, stream);
    if (e != cudaSuccess) {
        ftlm_batch_destroy_async(p, stream);
        return e == cudaErrorMemoryAllocation ? fail(FTLM_ENOMEM, "no device memory for a tuning run")
                                              : cuda_fail(e, "cudaMallocFromPoolAsync(tuning workspace)");
    }
    st = ftlm_batch_run(p, work, p->total, stream);
    if (st == FTLM_OK && (e = cudaEventRecord(ev[0], stream)) != cudaSuccess) st = cuda_fail(e, "event");
    if (st == FTLM_OK) st = ftlm_batch_run(p, work, p->total, stream);
    if (st == FTLM_OK && (e = cudaEventRecord(ev[1], stream)) != cudaSuccess) st = cuda_fail(e, "event");
    if (st == FTLM_OK && (e = cudaEventSynchronize(ev[1])) != cudaSuccess) st = cuda_fail(e, "tuning run");
    if (st == FTLM_OK && (e = cudaEventElapsedTime(ms, ev[0], ev[1])) != cudaSuccess)
        st = cuda_fail(e, "cudaEventElapsedTime");
    cudaFreeAsync(work, stream);
    ftlm_batch_destroy_async(p, stream);
    return st;
}

}  // namespace

extern "C" ftlm_status ftlm_batch_autotune_plan(int n, const ftlm_batch_item *items, int M, ftlm_vec_dist dist,
                                                ftlm_dtype dtype, void *stream_, ftlm_batch_plan *best,
                                                ftlm_batch_plan *tried, float *ms_out, int max_tried, int *n_tried)
{
    if (!best || !n_tried || max_tried < 0 || (max_tried > 0 && (!tried || !ms_out)))
        return fail(FTLM_EINVAL, "bad output arguments");
    cudaStream_t stream = (cudaStream_t)stream_;
    bool any_large = false, any_ms = false;
    for (int i = 0; i < n && items; ++i) {
        const ftlm_basis *b = items[i].basis;
        if (!b) continue;
        if (b->two_s == 1 && b->N > 32 && b->D > kSmallRows) any_large = true;
        if (b->two_s > 1 || (b->N <= 32 && b->D > kSmallRows)) any_ms = true;
    }
    int device = 0;
    cudaMemPool_t pool = nullptr;
    FTLM_CUDA(cudaGetDevice(&device));
    FTLM_CUDA(table_pool(device, &pool));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    FTLM_CUDA(cudaEventCreate(&ev[0]));
    FTLM_CUDA(cudaEventCreate(&ev[1]));
    ftlm_batch_plan cur{dtype == FTLM_F32 ? 16 : 8, any_large ? 4 : 1, (int)kMsTileRows, (int)kMsStreamRows};
    float cur_ms = -1.f;
    int count = 0;
    ftlm_status st = FTLM_OK;
    // coordinate search: block width (with the side-stream count where it matters),
    // then the H.v tile rows and the streaming tile rows of the multi-sector path
    auto consider = [&](const ftlm_batch_plan &cand) {
        float ms = 0.f;
        st = time_plan(n, items, M, dist, dtype, cand, stream, pool, ev, &ms);
        if (st != FTLM_OK) return;
        if (count < max_tried) {
            tried[count] = cand;
            ms_out[count] = ms;
        }
        ++count;
        if (cur_ms < 0.f || ms < cur_ms) {
            cur_ms = ms;
            cur = cand;
        }
    };
    for (int blk : {4, 8, 16})
        for (int sc : {1, 2, 4, 8}) {
            if (st != FTLM_OK || (!any_large && sc != 1)) break;
            ftlm_batch_plan c = cur;
            c.block = blk;
            c.streams = sc;
            consider(c);
        }
    if (any_ms) {
        const ftlm_batch_plan base = cur;
        for (int tr : {1024, 4096}) {
            if (st != FTLM_OK) break;
            ftlm_batch_plan c = base;
            c.tile_rows = tr;
            consider(c);
        }
        const ftlm_batch_plan base2 = cur;
        for (int sr : {8192, 32768}) {
            if (st != FTLM_OK) break;
            ftlm_batch_plan c = base2;
            c.stream_rows = sr;
            consider(c);
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != FTLM_OK) return st;
    *best = cur;
    *n_tried = count;
    return FTLM_OK;
}
