// Read-bandwidth probe for the roofline of the H.v kernels: a buffer that fits in
// L2 gives the L2 read rate the gathers are bounded by, a buffer far larger the
// DRAM read rate.  32 bytes per lane per load (the row of 8 FP32 or 4 FP64 values
// the block H.v gathers), coalesced, over `reps` passes in one launch.
#include "ftlm_internal.cuh"

namespace ftlm {

namespace {

__global__ void __launch_bounds__(256) read_probe_kernel(const uint4 *__restrict__ p, uint64_t n32, int reps,
                                                         unsigned int *sink)
{
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n32; i += stride) {
            const uint4 a = __ldg(p + 2 * i), b = __ldg(p + 2 * i + 1);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
        }
    if (acc == 0x9e3779b9u) *sink = acc;  // keeps the loads; practically never taken
}

}  // namespace

}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_probe_read_bandwidth(const void *buf_dev, uint64_t bytes, int reps, void *stream,
                                                 double *gbps)
{
    if (!buf_dev || !gbps || reps < 1 || bytes < 32) return fail(FTLM_EINVAL, "bad probe arguments");
    if ((uintptr_t)buf_dev & 31u) return fail(FTLM_EINVAL, "buffer must be 32-byte aligned");
    int dev = 0, sms = 0;
    FTLM_CUDA(cudaGetDevice(&dev));
    FTLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t n32 = bytes / 32;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FTLM_CUDA(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        // untimed pass (brings an L2-sized buffer into L2), then the timed passes
        read_probe_kernel<<<sms * 4, 256, 0, st>>>((const uint4 *)buf_dev, n32, 1, nullptr);
        note_launch();
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            read_probe_kernel<<<sms * 4, 256, 0, st>>>((const uint4 *)buf_dev, n32, reps, nullptr);
            note_launch();
            e = cudaEventRecord(e1, st);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) *gbps = (double)n32 * 32.0 * reps / (ms * 1e-3) / 1e9;
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "read probe");
    return FTLM_OK;
}
