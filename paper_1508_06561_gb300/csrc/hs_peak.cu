// hs_peak.cu -- integer issue-rate microbenchmarks for the scan's roofline.
//
// The scan is bound by integer instruction issue, not by HBM, so its
// roofline needs the GPU's integer throughput; a memory-copy rate or a
// tensor-core GEMM rate says nothing about it.  These kernels measure it:
// every thread runs eight interleaved dependency chains of one operation
// (each chain reads the next chain's latest value, so no result is dead and
// no two operations can be merged into one), enough warps are resident to
// hide the latency, and the rate is operations per second over the whole
// GPU, timed with CUDA events.  No counterpart in the paper.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hspeak.h"

namespace {

constexpr int kThreads = 1024;
constexpr int kUnroll = 8;              // rounds of the eight chains per loop trip

template <int kOp>
__device__ __forceinline__ uint32_t step(uint32_t a, uint32_t b, uint32_t c)
{
    if constexpr (kOp == HSP_IADD) return a + b;
    else if constexpr (kOp == HSP_DPX_MAX3) return (uint32_t)__vimax3_s32((int)a, (int)b, (int)c);
    else return (uint32_t)__viaddmax_s32((int)a, (int)b, (int)c);    // HSP_DPX_ADDMAX: max(a + b, c)
}

template <int kOp>
__global__ void __launch_bounds__(kThreads) peak_kernel(uint32_t *sink, int iters, uint32_t seed)
{
    uint32_t a0 = threadIdx.x ^ seed, a1 = a0 * 3u + 1u, a2 = a0 * 5u + 2u, a3 = a0 * 7u + 3u;
    uint32_t a4 = a0 * 11u + 4u, a5 = a0 * 13u + 5u, a6 = a0 * 17u + 6u, a7 = a0 * 19u + 7u;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            a0 = step<kOp>(a0, a1, a2);
            a1 = step<kOp>(a1, a2, a3);
            a2 = step<kOp>(a2, a3, a4);
            a3 = step<kOp>(a3, a4, a5);
            a4 = step<kOp>(a4, a5, a6);
            a5 = step<kOp>(a5, a6, a7);
            a6 = step<kOp>(a6, a7, a0);
            a7 = step<kOp>(a7, a0, a1);
        }
    }
    const uint32_t x = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
    if (x == seed) sink[blockIdx.x] = x;   // keeps the chains live; practically never taken
}

}  // namespace

extern "C" int hsp_ops_per_thread_trip(void) { return 8 * kUnroll; }

extern "C" int hsp_measure(int op, int iters, int reps, void *stream, double *ops_per_s, double *best_ms,
                           int64_t *ops_per_launch)
{
    if (!ops_per_s || !best_ms || !ops_per_launch || iters < 1 || reps < 1) return 1;
    if (op != HSP_IADD && op != HSP_DPX_MAX3 && op != HSP_DPX_ADDMAX) return 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
    void (*fn)(uint32_t *, int, uint32_t) =
        op == HSP_IADD ? peak_kernel<HSP_IADD> : op == HSP_DPX_MAX3 ? peak_kernel<HSP_DPX_MAX3> : peak_kernel<HSP_DPX_ADDMAX>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1) return 2;
    const int blocks = per_sm * sms;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaMalloc(&sink, sizeof(uint32_t) * blocks) != cudaSuccess) return 3;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = 2;
    float best = 1e30f;
    for (int r = -1; r < reps && rc == 0; r++) {      // r = -1: warm-up launch, not timed
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = 2; break; }
        fn<<<blocks, kThreads, 0, st>>>(sink, iters, 0x9E3779B9u + (uint32_t)r);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) { rc = 2; break; }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = 2; break; }
        if (r >= 0) best = std::min(best, ms);
    }
    if (rc == 0) {
        const int64_t ops = (int64_t)blocks * kThreads * (int64_t)iters * (8 * kUnroll);
        *ops_per_launch = ops;
        *best_ms = best;
        *ops_per_s = (double)ops / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
