// Error reporting and kernel timing shared by every entry point.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ftlm_internal.cuh"

namespace ftlm {

namespace {
thread_local std::string g_last_error;

struct ProfRecord {
    cudaEvent_t start, stop;
    int kind;
    int vectors;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_records;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
std::atomic<uint64_t> g_launches{0};
std::mutex g_pool_mu;
cudaMemPool_t g_pools[256] = {};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct OccKey {
    const void *kern;
    int threads;
    size_t smem;
    bool operator<(const OccKey &o) const
    {
        return kern != o.kern ? kern < o.kern : (threads != o.threads ? threads < o.threads : smem < o.smem);
    }
};
std::mutex g_occ_mu;
std::map<OccKey, int> g_occ;
}  // namespace

cudaError_t kernel_occupancy(const void *kern, int threads, size_t smem, bool set_smem_attr, int *occ)
{
    std::lock_guard<std::mutex> lk(g_occ_mu);
    const OccKey key{kern, threads, smem};
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
        *occ = it->second;
        return cudaSuccess;
    }
    cudaError_t e = cudaSuccess;
    if (set_smem_attr) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int v = 1;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem);
    if (e != cudaSuccess) return e;
    v = v < 1 ? 1 : v;
    g_occ[key] = v;
    *occ = v;
    return cudaSuccess;
}

cudaError_t table_pool(int device, cudaMemPool_t *pool)
{
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kPoolKeepBytes;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        // An allocation never waits for another stream: a block freed in the order of
        // a busy stream is taken only once that stream has passed the free (else the
        // pool grows), so that building tables or plans on a quiet stream does not
        // queue behind the Lanczos launches of a busy one.
        int no = 0;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseFollowEventDependencies, &no);
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[device] = p;
    }
    *pool = g_pools[device];
    return cudaSuccess;
}

namespace {

// Pinned staging for small host-to-device images (sector tables): a copy from
// pageable memory may wait until the stream's queued work has run, which blocks the
// host while the device is busy; a copy from a pinned buffer returns at once.  A
// ring of kUpStages buffers per device, each reused once its copy has run.
constexpr int kUpStages = 64;
constexpr size_t kUpStageBytes = 256 << 10;
struct UpRing {
    void *buf[kUpStages] = {};
    cudaEvent_t ev[kUpStages] = {};
    int next = 0;
};
std::mutex g_up_mu;
std::map<int, UpRing> g_up;

}  // namespace

cudaError_t upload_async(void *dst, const void *src, size_t bytes, cudaStream_t stream)
{
    if (bytes == 0) return cudaSuccess;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (bytes > kUpStageBytes) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
    std::lock_guard<std::mutex> lk(g_up_mu);
    UpRing &r = g_up[device];
    const int k = r.next;
    r.next = (r.next + 1) % kUpStages;
    if (!r.buf[k]) {
        e = cudaMallocHost(&r.buf[k], kUpStageBytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {  // no pinned memory: the pageable copy
            if (r.buf[k]) cudaFreeHost(r.buf[k]);
            r.buf[k] = nullptr;
            cudaGetLastError();
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
        }
    } else {
        e = cudaEventSynchronize(r.ev[k]);  // its previous copy has run
        if (e != cudaSuccess) return e;
    }
    std::memcpy(r.buf[k], src, bytes);
    e = cudaMemcpyAsync(dst, r.buf[k], bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(r.ev[k], stream);
    return e;
}

ftlm_status fail(ftlm_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

ftlm_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return FTLM_ECUDA;
}

void *profile_begin(int kind, cudaStream_t stream, int vectors)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return nullptr;
    ProfRecord r{take_event(), take_event(), kind, vectors};
    if (!r.start || !r.stop) return nullptr;
    if (cudaEventRecord(r.start, stream) != cudaSuccess) return nullptr;
    g_records.push_back(r);
    return reinterpret_cast<void *>(g_records.size());  // 1-based index
}

void profile_end(void *token, cudaStream_t stream)
{
    if (!token) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const size_t idx = reinterpret_cast<size_t>(token) - 1;
    if (idx < g_records.size()) cudaEventRecord(g_records[idx].stop, stream);
}

}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return FTLM_OK;
}

extern "C" ftlm_status ftlm_profile_read(uint64_t *hv_launches, uint64_t *hv_vectors, double *hv_ms,
                                         uint64_t *update_launches, double *update_ms)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    uint64_t n[2] = {0, 0}, vec = 0;
    double ms[2] = {0.0, 0.0};
    ftlm_status st = FTLM_OK;
    for (ProfRecord &r : g_records) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.start, r.stop);
        if (e != cudaSuccess && st == FTLM_OK) st = cuda_fail(e, "cudaEventElapsedTime");
        n[r.kind] += 1;
        ms[r.kind] += t;
        if (r.kind == kProfHv) vec += (uint64_t)r.vectors;
        g_event_pool.push_back(r.start);
        g_event_pool.push_back(r.stop);
    }
    g_records.clear();
    if (hv_launches) *hv_launches = n[kProfHv];
    if (hv_vectors) *hv_vectors = vec;
    if (hv_ms) *hv_ms = ms[kProfHv];
    if (update_launches) *update_launches = n[kProfUpdate];
    if (update_ms) *update_ms = ms[kProfUpdate];
    return st;
}

extern "C" ftlm_status ftlm_launch_count(uint64_t *count)
{
    if (!count) return fail(FTLM_EINVAL, "NULL argument");
    *count = g_launches.load(std::memory_order_relaxed);
    return FTLM_OK;
}

extern "C" const char *ftlm_status_string(ftlm_status s)
{
    switch (s) {
    case FTLM_OK: return "FTLM_OK";
    case FTLM_EINVAL: return "FTLM_EINVAL: invalid argument";
    case FTLM_ENOMEM: return "FTLM_ENOMEM: out of device memory or workspace too small";
    case FTLM_EUNSUPPORTED: return "FTLM_EUNSUPPORTED: outside what the library implements";
    case FTLM_ECUDA: return "FTLM_ECUDA: CUDA runtime error";
    case FTLM_ETIMEOUT: return "FTLM_ETIMEOUT: device wait expired";
    case FTLM_ENOCONV: return "FTLM_ENOCONV: a tridiagonal eigenproblem did not converge";
    }
    return "unknown ftlm_status";
}

extern "C" const char *ftlm_last_error(void) { return g_last_error.c_str(); }
