// Bandwidth ceilings for the roofline of the search kernel.
//
// The search's working set (node slots, registry, induced CSR) stays in the
// 129 MB L2, so its bandwidth ceiling is the L2 read rate, not HBM.  This
// file measures that rate with a plain read kernel: a buffer well inside L2
// is loaded once (warm-up), then read `reps` times per launch with 16-byte
// loads that bypass L1 (ld.global.cg), four independent loads in flight per
// thread per iteration, one block per SM times eight.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vc_gb300.h"

namespace {

__global__ void __launch_bounds__(512) l2_read_kernel(const uint4 *__restrict__ buf, long long nvec, int reps,
                                                      unsigned *sink)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned acc = 0;
    for (int r = 0; r < reps; r++) {
        long long i = tid;
        for (; i + 3 * nth < nvec; i += 4 * nth) {
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + nth), c = __ldcg(buf + i + 2 * nth),
                        d = __ldcg(buf + i + 3 * nth);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < nvec; i += nth) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;   // keeps the loads; the buffer is zero, so never taken
}

}  // namespace

extern "C" int vc_measure_l2_read(int64_t bytes, int32_t reps, int32_t trials, void *cuda_stream, double *gbs)
{
    if (!gbs || bytes < (1 << 20) || reps < 1 || trials < 1) return VC_EINVAL;
    *gbs = 0.0;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return VC_ECUDA;
    const long long nvec = bytes / 16;
    void *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)nvec * 16 + 256) != cudaSuccess) return VC_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = VC_OK;
    unsigned *sink = (unsigned *)((char *)buf + (size_t)nvec * 16);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, (size_t)nvec * 16 + 256, s) != cudaSuccess) {
        rc = VC_ECUDA;
    } else {
        const int blocks = 8 * sms, threads = 512;
        l2_read_kernel<<<blocks, threads, 0, s>>>((const uint4 *)buf, nvec, 1, sink);   // warm L2
        double best = 0.0;
        for (int t = 0; t < trials && rc == VC_OK; t++) {
            float ms = 0.f;
            if (cudaEventRecord(e0, s) != cudaSuccess) { rc = VC_ECUDA; break; }
            l2_read_kernel<<<blocks, threads, 0, s>>>((const uint4 *)buf, nvec, reps, sink);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = VC_ECUDA;
                break;
            }
            const double g = (double)nvec * 16.0 * reps / (ms * 1e-3) / 1e9;
            if (g > best) best = g;
        }
        *gbs = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    return rc;
}
