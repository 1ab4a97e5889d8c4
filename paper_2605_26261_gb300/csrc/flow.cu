// Continuous Lanczos flow: the chains of many sectors advance together, one H.v +
// update launch pair per Lanczos step for all of them, and sectors join and leave
// at step boundaries -- the chain-level continuous batching of a request loop.
//
// A sector's R chains are cut into units of B chains (the multi-sector units of
// msv.cu).  Each unit has its own region of the caller's workspace (two vector
// blocks, chain states, per-tile partial sums) and its own start launch j0: launch
// j of the flow runs the unit's Lanczos step j - j0, so a unit admitted while others
// are at step 40 starts at its step 1 in the same launch.  The units' rows are cut
// into the same tiles as in a batch and every unit reduces its own tiles in tile
// order, so a unit's results are bit-identical whether it runs alone or with any
// other units, and whenever it was admitted.  When a unit reaches its last step its
// chain lengths are copied out; the sectors whose units are all done get their Ritz
// step, one launch per step call on the flow's own stream (FP64 QR: slow on this
// GPU, so it overlaps the next call's Lanczos steps instead of delaying them), and
// their coefficient rows are reused once that launch has run.  Units are admitted while their regions fit in the
// workspace (first fit); a sector that does not fit is refused (FTLM_ENOMEM) and can
// be added again later.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ftlm_internal.cuh"
#include "msv.cuh"

namespace ftlm {

namespace {

uint64_t align256(uint64_t v) { return (v + 255) & ~255ull; }

// First-fit allocation of ranges of [0, capacity).
struct RangeAlloc {
    std::map<uint64_t, uint64_t> free_;  // offset -> length
    uint64_t free_total = 0;
    void init(uint64_t cap)
    {
        free_.clear();
        if (cap) free_[0] = cap;
        free_total = cap;
    }
    bool take(uint64_t len, uint64_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < len) continue;
            *off = it->first;
            const uint64_t rest = it->second - len, o = it->first + len;
            free_.erase(it);
            if (rest) free_[o] = rest;
            free_total -= len;
            return true;
        }
        return false;
    }
    void give(uint64_t off, uint64_t len)
    {
        if (!len) return;
        free_total += len;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct FlowUnit {
    MsUnit u;  // offsets into the unit region of the workspace; chain_base into the coefficient rows
    int kind;
    int item;
    uint64_t off, bytes;
    uint64_t vbytes;  // its two vector blocks (the wave budget counts these)
    int done;         // Lanczos steps completed
};

struct FlowItem {
    ftlm_batch_item it;
    int ticket;
    int units_left;
    uint32_t chain_base;
    bool live;
};

// A wave stream of the flow and the event that joins it back to the caller's.
struct FlowSlot {
    cudaStream_t s;
    cudaEvent_t join;
};
constexpr int kFlowSlots = 4;      // wave streams at most
constexpr int kFlowSlotsDefault = 4;

int kind_of(const ftlm_basis *b) { return b->two_s > 1 ? kMsSpin : (b->mode == FTLM_RANK_CLT ? kMsClt : kMsCr); }

// Region of one unit of B chains of b: two vector blocks, states and counter, and
// the per-tile partial sums (H.v tiles outnumber the streaming tiles).
uint64_t unit_bytes(const ftlm_basis *b, int B, uint64_t vsize)
{
    const uint64_t vb = align256(b->D * (uint64_t)B * vsize);
    const uint64_t nt = (b->D + kMsTileRows - 1) / kMsTileRows;
    return 2 * vb + align256(kMaxBlock * sizeof(ChainState) + 64) + align256(nt * B * sizeof(double));
}

__global__ void flow_meff_kernel(const MsUnit *__restrict__ units, const uint32_t *__restrict__ fin, uint32_t n,
                                 int B, int *meff, char *ws)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n * (uint32_t)B; i += gridDim.x * blockDim.x) {
        const MsUnit &U = units[fin[i / B]];
        const int r = (int)(i % B);
        if (r < U.nact) meff[U.chain_base + r] = reinterpret_cast<const ChainState *>(ws + U.off_st)[r].m_eff;
    }
}

}  // namespace

}  // namespace ftlm

struct ftlm_flow {
    ftlm_dtype dtype;
    int B, M, dist, num_sms, device;
    uint32_t max_units, max_chains;
    // caller workspace: [alpha | beta : max_chains x M doubles][meff : max_chains ints][unit regions]
    char *work;
    double *alpha, *beta;
    int *meff;
    char *units_base;  // start of the unit regions (the ws of the msv kernels)
    uint64_t units_bytes;
    ftlm::RangeAlloc region, chains;
    // device descriptors of a step call's waves: units, per-kind H.v tile maps,
    // streaming tile map, finished lists; and the Ritz rows
    void *dev_block;
    ftlm::MsUnit *d_units;
    uint32_t *d_tile[3], *d_stile, *d_fin;
    ftlm::FlowSlot slot[ftlm::kFlowSlots];
    int n_slots;           // wave streams in use (ftlm_flow_set_streams)
    cudaEvent_t ev_fork;   // the caller's stream at the start of a step call
    ftlm::RitzRow *d_ritz;
    // the Ritz launches: own stream, the event it waits for on the caller's stream,
    // the event after its latest launch, and the coefficient rows (offset, count)
    // still read by a queued launch
    cudaStream_t rz;
    cudaEvent_t ev_main, ev_rz;
    std::vector<std::pair<uint64_t, uint64_t>> rows_pending;
    uint64_t cap_tiles, cap_stiles;
    // pinned staging for the uploads (a ring of buffers, each reused once its copies ran)
    static constexpr int kStages = 8;
    char *stage[kStages];
    cudaEvent_t stage_ev[kStages];
    uint64_t stage_bytes;
    int stage_cur;
    std::vector<ftlm::FlowUnit> units;
    std::vector<ftlm::FlowItem> items;
    std::vector<int> done;  // tickets whose outputs are queued
    int next_ticket;
    uint64_t wave_bytes;  // vector bytes per wave
};

using namespace ftlm;

namespace {

// The next pinned staging buffer (waits until its previous copies have run).
ftlm_status stage_next(ftlm_flow *f, char **buf)
{
    f->stage_cur = (f->stage_cur + 1) % ftlm_flow::kStages;
    FTLM_CUDA(cudaEventSynchronize(f->stage_ev[f->stage_cur]));
    *buf = f->stage[f->stage_cur];
    return FTLM_OK;
}

// One wave of a step call: its units (indices into f->units) in descriptor order,
// grouped by rank kind, and where its descriptors, tile maps and finished list sit
// in the call's upload.  A unit's launches run as step j - j0 with j0 = -done, so
// launch j = 1, 2, ... of the wave is the unit's step done + j.
struct WavePlan {
    std::vector<uint32_t> order;
    uint32_t unit0;                       // first descriptor of the wave
    uint32_t kind_first[3], kind_count[3];  // descriptor ranges per kind (wave-local)
    uint32_t tile0[3], n_tiles[3];        // ranges of the kinds' H.v tile maps
    uint32_t stile0, n_stiles;            // range of the streaming tile map
    uint32_t fin0, n_fin;                 // wave-local positions of units that finish
    int steps;                            // Lanczos steps of this call
    bool fresh;                           // some unit starts now
    uint64_t load;                        // rows x steps
};

// Plans of the waves (consecutive units in admission order, at most wave_bytes of
// vectors each) and their descriptors, tile maps and finished lists, uploaded to
// the device in one copy per array on `stream`.
ftlm_status plan_waves(ftlm_flow *f, int steps, std::vector<WavePlan> &waves, cudaStream_t stream)
{
    std::vector<std::vector<uint32_t>> groups;
    uint64_t wb = 0;
    for (uint32_t i = 0; i < f->units.size(); ++i) {
        const FlowUnit &u = f->units[i];
        if (groups.empty() || wb + u.vbytes > f->wave_bytes) {
            groups.emplace_back();
            wb = 0;
        }
        groups.back().push_back(i);
        wb += u.vbytes;
    }
    std::vector<MsUnit> du;
    std::vector<uint32_t> tiles[3], stiles, fins;
    waves.assign(groups.size(), WavePlan{});
    for (size_t w = 0; w < groups.size(); ++w) {
        WavePlan &p = waves[w];
        p.unit0 = (uint32_t)du.size();
        for (int kind = 0; kind < 3; ++kind) {
            p.kind_first[kind] = (uint32_t)p.order.size();
            for (uint32_t i : groups[w])
                if (f->units[i].kind == kind) p.order.push_back(i);
            p.kind_count[kind] = (uint32_t)p.order.size() - p.kind_first[kind];
            p.tile0[kind] = (uint32_t)tiles[kind].size();
        }
        p.stile0 = (uint32_t)stiles.size();
        p.fin0 = (uint32_t)fins.size();
        int need = 0;
        for (uint32_t i : p.order) need = std::max(need, f->units[i].u.m_max - f->units[i].done);
        p.steps = std::min(steps, need);
        for (uint32_t pos = 0; pos < p.order.size(); ++pos) {
            const FlowUnit &fu = f->units[p.order[pos]];
            MsUnit u = fu.u;
            const int kind = fu.kind;
            u.j0 = -fu.done;
            u.tile0 = (uint32_t)tiles[kind].size() - p.tile0[kind];
            for (uint32_t k = 0; k < u.n_tiles; ++k) tiles[kind].push_back(pos - p.kind_first[kind]);  // kind-local
            u.stile0 = (uint32_t)stiles.size() - p.stile0;
            for (uint32_t k = 0; k < u.n_stiles; ++k) stiles.push_back(pos);  // wave-local
            du.push_back(u);
            p.fresh |= fu.done == 0;
            if (fu.done + p.steps >= fu.u.m_max) fins.push_back(pos);
            p.load += fu.u.s.D * (uint64_t)std::max(0, std::min(p.steps, fu.u.m_max - fu.done));
        }
        for (int kind = 0; kind < 3; ++kind) p.n_tiles[kind] = (uint32_t)tiles[kind].size() - p.tile0[kind];
        p.n_stiles = (uint32_t)stiles.size() - p.stile0;
        p.n_fin = (uint32_t)fins.size() - p.fin0;
    }
    for (int kind = 0; kind < 3; ++kind)
        if (tiles[kind].size() > f->cap_tiles) return fail(FTLM_ENOMEM, "flow tile map full");
    if (stiles.size() > f->cap_stiles) return fail(FTLM_ENOMEM, "flow tile map full");
    char *buf = nullptr;
    ftlm_status st = stage_next(f, &buf);
    if (st != FTLM_OK) return st;
    uint64_t off = 0;
    auto put = [&](void *dst, const void *src, uint64_t bytes) -> cudaError_t {
        if (!bytes) return cudaSuccess;
        std::memcpy(buf + off, src, bytes);
        const cudaError_t e = cudaMemcpyAsync(dst, buf + off, bytes, cudaMemcpyHostToDevice, stream);
        off = align256(off + bytes);
        return e;
    };
    FTLM_CUDA(put(f->d_units, du.data(), du.size() * sizeof(MsUnit)));
    for (int kind = 0; kind < 3; ++kind)
        FTLM_CUDA(put(f->d_tile[kind], tiles[kind].data(), tiles[kind].size() * sizeof(uint32_t)));
    FTLM_CUDA(put(f->d_stile, stiles.data(), stiles.size() * sizeof(uint32_t)));
    FTLM_CUDA(put(f->d_fin, fins.data(), fins.size() * sizeof(uint32_t)));
    FTLM_CUDA(cudaEventRecord(f->stage_ev[f->stage_cur], stream));
    return FTLM_OK;
}

// The launches of one wave on `stream`: start vectors of its new units, then per
// step one H.v launch per rank kind and one update launch, then the chain lengths
// of its units that reach their last step.  Appends to fin the indices (into
// f->units) of those units and to ritz the sectors whose units are all done.
ftlm_status run_wave(ftlm_flow *f, const WavePlan &p, cudaStream_t stream, std::vector<uint32_t> &fin,
                     std::vector<int> &ritz)
{
    const MsUnit *units = f->d_units + p.unit0;
    const uint32_t *stile = f->d_stile + p.stile0;
    const uint32_t n_units = (uint32_t)p.order.size();
    ftlm_status s;
    if (p.fresh) {  // units with j0 == 0: reset and start vectors
        s = ms_flow_start(f->dtype, f->B, units, n_units, stile, p.n_stiles, 0, f->dist, f->units_base, f->num_sms,
                          stream);
        if (s != FTLM_OK) return s;
    }
    for (int j = 1; j <= p.steps; ++j) {
        for (int kind = 0; kind < 3; ++kind) {
            if (!p.kind_count[kind]) continue;
            s = ms_flow_hv(f->dtype, f->B, kind, units + p.kind_first[kind], f->d_tile[kind] + p.tile0[kind],
                           p.n_tiles[kind], j, f->M, f->alpha, f->units_base, f->num_sms, stream);
            if (s != FTLM_OK) return s;
        }
        s = ms_flow_update(f->dtype, f->B, units, stile, p.n_stiles, j, f->M, f->beta, f->units_base, f->num_sms,
                           stream);
        if (s != FTLM_OK) return s;
    }
    if (p.n_fin) {
        flow_meff_kernel<<<(unsigned)((p.n_fin * f->B + 255) / 256), 256, 0, stream>>>(
            units, f->d_fin + p.fin0, p.n_fin, f->B, f->meff, f->units_base);
        note_launch();
        FTLM_CUDA(cudaGetLastError());
    }
    for (uint32_t i : p.order) {
        FlowUnit &u = f->units[i];
        u.done = std::min(u.u.m_max, u.done + p.steps);
        if (u.done < u.u.m_max) continue;
        fin.push_back(i);
        f->region.give(u.off, u.bytes);
        FlowItem &it = f->items[u.item];
        if (--it.units_left == 0) ritz.push_back(u.item);
    }
    return FTLM_OK;
}

// One Ritz launch on the flow's stream for the sectors (indices into f->items) that
// finished in this step call, after the call's work on `stream`; their chain rows
// are released once that launch has run (release_rows).
ftlm_status queue_ritz(ftlm_flow *f, const std::vector<int> &items, cudaStream_t stream)
{
    if (items.empty()) return FTLM_OK;
    std::vector<RitzRow> rows;
    for (int k : items) {
        const ftlm_batch_item &bi = f->items[k].it;
        for (int r = 0; r < bi.R; ++r) {
            RitzRow w{};
            w.theta = bi.theta_dev + (size_t)r * f->M;
            w.weight = bi.weight_dev + (size_t)r * f->M;
            w.m_eff = bi.m_eff_dev + r;
            w.row = f->items[k].chain_base + (uint32_t)r;
            rows.push_back(w);
        }
    }
    FTLM_CUDA(cudaEventRecord(f->ev_main, stream));
    FTLM_CUDA(cudaStreamWaitEvent(f->rz, f->ev_main, 0));
    char *buf = nullptr;
    ftlm_status s = stage_next(f, &buf);
    if (s != FTLM_OK) return s;
    std::memcpy(buf, rows.data(), rows.size() * sizeof(RitzRow));
    // the rows buffer is only written and read on the Ritz stream, in order
    FTLM_CUDA(cudaMemcpyAsync(f->d_ritz, buf, rows.size() * sizeof(RitzRow), cudaMemcpyHostToDevice, f->rz));
    FTLM_CUDA(cudaEventRecord(f->stage_ev[f->stage_cur], f->rz));
    s = launch_ritz_rows((int)rows.size(), f->M, f->alpha, f->beta, f->meff, f->d_ritz, f->rz);
    if (s != FTLM_OK) return s;
    FTLM_CUDA(cudaEventRecord(f->ev_rz, f->rz));
    for (int k : items) {
        FlowItem &it = f->items[k];
        f->rows_pending.emplace_back(it.chain_base, (uint64_t)it.it.R);
        f->done.push_back(it.ticket);
        it.live = false;
    }
    return FTLM_OK;
}

// Coefficient rows of finished sectors back to the free list once the Ritz launches
// that read them have run (wait: block the host until they have).
ftlm_status release_rows(ftlm_flow *f, bool wait)
{
    if (f->rows_pending.empty()) return FTLM_OK;
    if (wait) {
        FTLM_CUDA(cudaEventSynchronize(f->ev_rz));
    } else {
        const cudaError_t e = cudaEventQuery(f->ev_rz);
        if (e == cudaErrorNotReady) return FTLM_OK;
        FTLM_CUDA(e);
    }
    for (const auto &p : f->rows_pending) f->chains.give(p.first, p.second);
    f->rows_pending.clear();
    return FTLM_OK;
}

}  // namespace

extern "C" ftlm_status ftlm_flow_unit_bytes(const ftlm_basis *b, ftlm_dtype dtype, int block, uint64_t *bytes)
{
    if (!b || !bytes) return fail(FTLM_EINVAL, "NULL argument");
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    if (!valid_block(block)) return fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    *bytes = unit_bytes(b, block, dtype == FTLM_F32 ? 4 : 8);
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_flow_create(ftlm_dtype dtype, int block, int M, ftlm_vec_dist dist, int max_units,
                                        void *work_dev, uint64_t work_bytes, void *stream_, ftlm_flow **out)
{
    if (!out) return fail(FTLM_EINVAL, "out is NULL");
    *out = nullptr;
    if (dtype != FTLM_F32 && dtype != FTLM_F64) return fail(FTLM_EINVAL, "bad dtype");
    if (!valid_block(block)) return fail(FTLM_EINVAL, "block width must be 1, 4, 8 or 16");
    if (M < 1 || M > FTLM_MAX_LANCZOS) return fail(FTLM_EINVAL, "M out of range");
    if (dist != FTLM_VEC_GAUSS && dist != FTLM_VEC_RADEMACHER) return fail(FTLM_EINVAL, "bad distribution");
    if (max_units < 1 || max_units > (1 << 20)) return fail(FTLM_EINVAL, "max_units out of range");
    if (!work_dev || ((uintptr_t)work_dev & 255u)) return fail(FTLM_EINVAL, "workspace NULL or not 256-byte aligned");
    cudaStream_t stream = (cudaStream_t)stream_;
    ftlm_flow *f = new (std::nothrow) ftlm_flow();
    if (!f) return fail(FTLM_ENOMEM, "host allocation failed");
    f->dtype = dtype;
    f->B = block;
    f->M = M;
    f->dist = dist;
    f->max_units = (uint32_t)max_units;
    f->max_chains = (uint32_t)max_units * (uint32_t)block;
    const uint64_t coef = align256((uint64_t)f->max_chains * M * sizeof(double));
    const uint64_t head = 2 * coef + align256((uint64_t)f->max_chains * sizeof(int));
    if (work_bytes <= head) {
        delete f;
        return fail(FTLM_ENOMEM, "workspace smaller than the coefficient rows of max_units units");
    }
    f->work = (char *)work_dev;
    f->alpha = (double *)f->work;
    f->beta = (double *)(f->work + coef);
    f->meff = (int *)(f->work + 2 * coef);
    f->units_base = f->work + head;
    f->units_bytes = work_bytes - head;
    f->region.init(f->units_bytes);
    f->chains.init(f->max_chains);
    f->next_ticket = 1;
    f->wave_bytes = ms_wave_bytes();
    cudaError_t e = cudaGetDevice(&f->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, f->device);
    if (e != cudaSuccess) {
        delete f;
        return cuda_fail(e, "cudaGetDevice");
    }
    // tile maps: every unit row needs 2 B values of vectors at least
    const uint64_t rows = f->units_bytes / (2ull * block * (dtype == FTLM_F32 ? 4 : 8));
    f->cap_tiles = rows / kMsTileRows + max_units + 1;
    f->cap_stiles = rows / kMsStreamRows + max_units + 1;
    // [units | 3 H.v tile maps | streaming map | finished lists | Ritz rows]; the
    // tiles of every unit together number at most cap_tiles (cap_stiles)
    const uint64_t o_units = 0;
    const uint64_t o_tile = align256((uint64_t)max_units * sizeof(MsUnit));
    const uint64_t o_stile = o_tile + 3 * align256(f->cap_tiles * sizeof(uint32_t));
    const uint64_t o_fin = o_stile + align256(f->cap_stiles * sizeof(uint32_t));
    const uint64_t o_ritz = o_fin + align256((uint64_t)max_units * sizeof(uint32_t));
    const uint64_t total = o_ritz + align256((uint64_t)f->max_chains * sizeof(RitzRow));
    cudaMemPool_t pool = nullptr;
    e = table_pool(f->device, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&f->dev_block, total, pool, stream);
    if (e != cudaSuccess) {
        delete f;
        return e == cudaErrorMemoryAllocation ? fail(FTLM_ENOMEM, "no device memory for the flow descriptors")
                                              : cuda_fail(e, "cudaMallocFromPoolAsync(flow)");
    }
    // pinned staging: the descriptors, tile maps (of all kinds together at most
    // cap_tiles) and finished lists of a step call's waves, or its Ritz rows
    f->stage_bytes = std::max<uint64_t>(o_tile + align256(f->cap_tiles * sizeof(uint32_t)) +
                                            align256(f->cap_stiles * sizeof(uint32_t)) +
                                            align256((uint64_t)max_units * sizeof(uint32_t)) + 6 * 256,
                                        total - o_ritz);
    f->n_slots = kFlowSlotsDefault;
    f->ev_fork = nullptr;
    for (int k = 0; k < kFlowSlots; ++k) {
        f->slot[k].s = nullptr;
        f->slot[k].join = nullptr;
    }
    for (int k = 0; k < ftlm_flow::kStages; ++k) {
        f->stage[k] = nullptr;
        f->stage_ev[k] = nullptr;
    }
    f->stage_cur = 0;
    f->rz = nullptr;
    f->ev_main = f->ev_rz = nullptr;
    for (int k = 0; k < ftlm_flow::kStages && e == cudaSuccess; ++k) {
        e = cudaMallocHost((void **)&f->stage[k], f->stage_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->stage_ev[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->rz, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_main, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_rz, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming);
    for (int k = 0; k < kFlowSlots && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&f->slot[k].s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->slot[k].join, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        for (int k = 0; k < ftlm_flow::kStages; ++k) {
            if (f->stage[k]) cudaFreeHost(f->stage[k]);
            if (f->stage_ev[k]) cudaEventDestroy(f->stage_ev[k]);
        }
        if (f->rz) cudaStreamDestroy(f->rz);
        if (f->ev_main) cudaEventDestroy(f->ev_main);
        if (f->ev_rz) cudaEventDestroy(f->ev_rz);
        if (f->ev_fork) cudaEventDestroy(f->ev_fork);
        for (int k = 0; k < kFlowSlots; ++k) {
            if (f->slot[k].s) cudaStreamDestroy(f->slot[k].s);
            if (f->slot[k].join) cudaEventDestroy(f->slot[k].join);
        }
        cudaFreeAsync(f->dev_block, stream);
        delete f;
        return cuda_fail(e, "flow staging buffers and streams");
    }
    char *base = (char *)f->dev_block;
    f->d_units = (MsUnit *)(base + o_units);
    for (int k = 0; k < 3; ++k) f->d_tile[k] = (uint32_t *)(base + o_tile + k * align256(f->cap_tiles * sizeof(uint32_t)));
    f->d_stile = (uint32_t *)(base + o_stile);
    f->d_fin = (uint32_t *)(base + o_fin);
    f->d_ritz = (RitzRow *)(base + o_ritz);
    *out = f;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_flow_add(ftlm_flow *f, const ftlm_batch_item *item, int *ticket)
{
    if (!f || !item || !ticket) return fail(FTLM_EINVAL, "NULL argument");
    const ftlm_basis *b = item->basis;
    if (!b || item->R < 1 || item->first_chain < 0) return fail(FTLM_EINVAL, "bad item");
    if (!item->theta_dev || !item->weight_dev || !item->m_eff_dev) return fail(FTLM_EINVAL, "NULL output in item");
    if (b->two_s == 1 && b->N > 32) return fail(FTLM_EUNSUPPORTED, "flow sectors need N <= 32 at s = 1/2");
    if (b->device != f->device) return fail(FTLM_EINVAL, "basis on another device");
    const int B = f->B;
    const uint64_t vsize = f->dtype == FTLM_F32 ? 4 : 8;
    const int nu = (item->R + B - 1) / B;
    if (f->units.size() + nu > f->max_units) return fail(FTLM_ENOMEM, "flow holds max_units units");
    uint64_t cb = 0;
    if (!f->chains.take((uint64_t)item->R, &cb)) {
        // rows held only by queued Ritz launches: wait for those
        if (f->rows_pending.empty()) return fail(FTLM_ENOMEM, "no coefficient rows free");
        ftlm_status s = release_rows(f, true);
        if (s != FTLM_OK) return s;
        if (!f->chains.take((uint64_t)item->R, &cb)) return fail(FTLM_ENOMEM, "no coefficient rows free");
    }
    const uint64_t ub = unit_bytes(b, B, vsize);
    std::vector<uint64_t> offs;
    for (int k = 0; k < nu; ++k) {
        uint64_t off = 0;
        if (!f->region.take(ub, &off)) {
            for (uint64_t o : offs) f->region.give(o, ub);
            f->chains.give(cb, (uint64_t)item->R);
            return fail(FTLM_ENOMEM, "the flow workspace has no room for this sector now");
        }
        offs.push_back(off);
    }
    FlowItem it{};
    it.it = *item;
    it.ticket = f->next_ticket++;
    it.units_left = nu;
    it.chain_base = (uint32_t)cb;
    it.live = true;
    const int idx = (int)f->items.size();
    f->items.push_back(it);
    const uint64_t vb = align256(b->D * (uint64_t)B * vsize);
    for (int k = 0; k < nu; ++k) {
        const int r0 = k * B;
        FlowUnit fu{};
        MsUnit &u = fu.u;
        u.s = b->tables();
        u.bl = b->mode == FTLM_RANK_CLT ? b->bonds_clt : b->bonds_cr;
        u.spin = b->spin;
        u.off_v0 = offs[k];
        u.off_v1 = offs[k] + vb;
        u.off_st = offs[k] + 2 * vb;
        u.off_part = u.off_st + align256(kMaxBlock * sizeof(ChainState) + 64);
        u.seed = item->seed;
        u.tau = f->dtype == FTLM_F32 ? b->tau32 : b->tau64;
        u.tile_rows = kMsTileRows;
        u.stream_rows = kMsStreamRows;
        u.n_tiles = (uint32_t)((b->D + kMsTileRows - 1) / kMsTileRows);
        u.n_stiles = (uint32_t)((b->D + kMsStreamRows - 1) / kMsStreamRows);
        u.chain_base = (uint32_t)cb + (uint32_t)r0;
        u.key_n = b->key_n;
        u.K = b->K;
        u.chain0 = item->first_chain + r0;
        u.nact = std::min(B, item->R - r0);
        u.m_max = (uint64_t)f->M < b->D ? f->M : (int)b->D;
        fu.kind = kind_of(b);
        fu.item = idx;
        fu.off = offs[k];
        fu.bytes = ub;
        fu.vbytes = 2 * vb;
        fu.done = 0;
        f->units.push_back(fu);
    }
    *ticket = it.ticket;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_flow_step(ftlm_flow *f, int steps, void *stream_)
{
    if (!f || steps < 0) return fail(FTLM_EINVAL, "bad flow step");
    cudaStream_t stream = (cudaStream_t)stream_;
    ftlm_status st = release_rows(f, false);
    if (st != FTLM_OK) return st;
    if (!steps || f->units.empty()) return FTLM_OK;
    // the sectors that start now: coefficient rows to zero
    for (const FlowUnit &u : f->units)
        if (u.done == 0 && u.u.chain_base == f->items[u.item].chain_base) {
            const FlowItem &it = f->items[u.item];
            const size_t rows = (size_t)it.it.R * f->M * sizeof(double);
            FTLM_CUDA(cudaMemsetAsync(f->alpha + (size_t)it.chain_base * f->M, 0, rows, stream));
            FTLM_CUDA(cudaMemsetAsync(f->beta + (size_t)it.chain_base * f->M, 0, rows, stream));
        }
    std::vector<WavePlan> waves;
    st = plan_waves(f, steps, waves, stream);
    if (st != FTLM_OK) return st;
    // each wave on the least loaded wave stream (the waves of one stream run in
    // order); the wave streams start after the caller's stream (the upload above)
    // and it waits for them
    const int ns = std::min<int>(f->n_slots, (int)waves.size());
    std::vector<uint64_t> load(ns, 0);
    std::vector<int> slot_of(waves.size(), 0);
    for (size_t w = 0; w < waves.size(); ++w) {
        const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        slot_of[w] = q;
        load[q] += waves[w].load;
    }
    if (ns > 1) {
        FTLM_CUDA(cudaEventRecord(f->ev_fork, stream));
        for (int q = 0; q < ns; ++q) FTLM_CUDA(cudaStreamWaitEvent(f->slot[q].s, f->ev_fork, 0));
    }
    std::vector<uint32_t> fin;
    std::vector<int> ritz;
    for (size_t w = 0; w < waves.size(); ++w) {
        st = run_wave(f, waves[w], ns > 1 ? f->slot[slot_of[w]].s : stream, fin, ritz);
        if (st != FTLM_OK) return st;
    }
    if (ns > 1)
        for (int q = 0; q < ns; ++q) {
            FTLM_CUDA(cudaEventRecord(f->slot[q].join, f->slot[q].s));
            FTLM_CUDA(cudaStreamWaitEvent(stream, f->slot[q].join, 0));
        }
    if (!fin.empty()) {
        std::vector<bool> gone(f->units.size(), false);
        for (uint32_t i : fin) gone[i] = true;
        std::vector<FlowUnit> keep;
        for (uint32_t i = 0; i < f->units.size(); ++i)
            if (!gone[i]) keep.push_back(f->units[i]);
        f->units = keep;
    }
    return queue_ritz(f, ritz, stream);
}

extern "C" ftlm_status ftlm_flow_set_streams(ftlm_flow *f, int n)
{
    if (!f) return fail(FTLM_EINVAL, "NULL flow");
    if (n < 1 || n > kFlowSlots) return fail(FTLM_EINVAL, "wave streams must be 1 .. 4");
    f->n_slots = n;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_flow_wait_outputs(ftlm_flow *f, void *stream)
{
    if (!f) return fail(FTLM_EINVAL, "NULL flow");
    FTLM_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, f->ev_rz, 0));
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_flow_done(ftlm_flow *f, int *tickets, int max, int *n)
{
    if (!f || !n || max < 0 || (max > 0 && !tickets)) return fail(FTLM_EINVAL, "bad argument");
    const int k = std::min<int>(max, (int)f->done.size());
    for (int i = 0; i < k; ++i) tickets[i] = f->done[i];
    f->done.erase(f->done.begin(), f->done.begin() + k);
    *n = k;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_flow_status(const ftlm_flow *f, int *units, int *items, uint64_t *free_bytes)
{
    if (!f) return fail(FTLM_EINVAL, "NULL flow");
    if (units) *units = (int)f->units.size();
    if (items) {
        int live = 0;
        for (const FlowItem &it : f->items) live += it.live ? 1 : 0;
        *items = live;
    }
    if (free_bytes) *free_bytes = f->region.free_total;
    return FTLM_OK;
}

extern "C" void ftlm_flow_destroy(ftlm_flow *f)
{
    if (!f) return;
    cudaDeviceSynchronize();
    cudaFreeAsync(f->dev_block, 0);
    for (int k = 0; k < ftlm_flow::kStages; ++k) {
        cudaFreeHost(f->stage[k]);
        cudaEventDestroy(f->stage_ev[k]);
    }
    cudaStreamDestroy(f->rz);
    cudaEventDestroy(f->ev_main);
    cudaEventDestroy(f->ev_rz);
    cudaEventDestroy(f->ev_fork);
    for (int k = 0; k < kFlowSlots; ++k) {
        cudaStreamDestroy(f->slot[k].s);
        cudaEventDestroy(f->slot[k].join);
    }
    delete f;
}
