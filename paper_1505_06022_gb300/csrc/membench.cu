// membench.cu -- read bandwidth of one memory tier, the denominator of the traversal's roofline.
//
// A plain streaming read over a device buffer, L1 bypassed (ld.global.cg), 16-byte loads,
// four in flight per thread, one resident grid. With a buffer well below the L2 capacity
// (129 MB on GB300) and a warm-up pass first, every timed load is an L2 hit: the rate is what the
// L2 can deliver to the SMs. With a buffer many times the L2 it is the HBM read rate.
#include <string>

#include "gsp_internal.h"

namespace {

__global__ void __launch_bounds__(512) k_read_stream(const uint4* __restrict__ p, int64_t n, int32_t reps,
                                                     uint32_t* __restrict__ sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int32_t r = 0; r < reps; ++r) {
        int64_t i = start;
        for (; i + 3 * stride < n; i += 4 * stride) {
            const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride);
            const uint4 c = __ldcg(p + i + 2 * stride), d = __ldcg(p + i + 3 * stride);
            acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^ (d.x ^ d.y ^ d.z ^ d.w);
        }
        for (; i < n; i += stride) {
            const uint4 a = __ldcg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    // the buffer is zero-filled, so this never stores; the compiler cannot know that and keeps
    // every load
    if (acc == 0x2545F491u) sink[start & 255] = acc;
}

}  // namespace

extern "C" gsp_status gsp_measure_read_bandwidth(gsp_context* ctx, int64_t bytes, int32_t reps, double* gbps) {
    if (!ctx || !gbps || bytes < 16 * 1024 || (bytes & 15) || reps < 1) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(ctx->device));
    GSP_NO_PENDING_ERROR("gsp_measure_read_bandwidth");
    int sms = 0;
    GSP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    uint4* buf = nullptr;
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, (size_t)bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 256 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, (size_t)bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        const int64_t n = bytes / 16;
        const int grid = sms * 4;  // 2,048 threads per SM
        k_read_stream<<<grid, 512>>>(buf, n, 1, sink);  // warm-up: brings a small buffer into L2
        cudaEventRecord(e0);
        k_read_stream<<<grid, 512>>>(buf, n, reps, sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (e != cudaSuccess) {
        const gsp_status st = gsp_cuda_fail(e);
        gsp_set_last_error(std::string("gsp_measure_read_bandwidth: ") + cudaGetErrorString(e));
        return st;
    }
    *gbps = (double)bytes * (double)reps / ((double)ms * 1e-3) / 1e9;
    return GSP_OK;
}
