// hs_topk.cu -- ranking of the scanned pairs (Sec. IV: results ranked by
// score; read as the k best).  Order: score descending, then database index
// ascending.  Each pair becomes the 64-bit key
//     ((score ^ 0x80000000) << 32) | (0xFFFFFFFF - index)
// so a larger key is a better hit and all keys are distinct.  Every CTA
// selects the k largest keys of its slice with an MSB-first radix select in
// shared memory; the last CTA to finish selects the k largest of those
// candidates, sorts them and writes the ranked (index, score) list.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr int kSortMax = HS_MAX_K;     // bitonic sort buffer (keys)

struct ScoreKeys {      // the slice [lo, lo+m) of the score array
    const int32_t *scores;
    int64_t lo;
    __device__ __forceinline__ uint64_t operator()(int64_t i) const
    {
        const uint32_t s = (uint32_t)((volatile const int32_t *)scores)[lo + i] ^ 0x80000000u;
        return ((uint64_t)s << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)(lo + i));
    }
};

struct CandKeys {       // candidates written by the other CTAs (0 = empty slot)
    const uint64_t *cand;
    __device__ __forceinline__ uint64_t operator()(int64_t i) const
    {
        return ((volatile const uint64_t *)cand)[i];
    }
};

struct SelectSmem {
    uint32_t hist[256];
    uint32_t suffix[257];
    uint64_t prefix, mask;
    uint32_t remaining;
    uint32_t count;
};

// Exact k-th largest key among m keys (k <= m), by 8 passes of 8 bits.
template <class Keys>
__device__ uint64_t radix_kth(const Keys &key, int64_t m, uint32_t k, SelectSmem &sm)
{
    if (threadIdx.x == 0) { sm.prefix = 0; sm.mask = 0; sm.remaining = k; }
    __syncthreads();
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) sm.hist[b] = 0;
        __syncthreads();
        const uint64_t prefix = sm.prefix, mask = sm.mask;
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
            const uint64_t x = key(i);
            if (x != 0 && (x & mask) == prefix) atomicAdd(&sm.hist[(x >> shift) & 255u], 1u);
        }
        __syncthreads();
        // suffix[b] = number of candidate keys whose digit is >= b
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            // lane l owns bins 8l .. 8l+7 (descending within the warp scan)
            uint32_t local[8];
            uint32_t tot = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) { local[j] = sm.hist[8 * lane + j]; tot += local[j]; }
            // suffix over lanes: sum of tot of lanes > l
            uint32_t incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_down_sync(0xFFFFFFFFu, incl, o);
                if (lane + o < 32) incl += y;
            }
            uint32_t run = incl - tot;     // keys in bins above this lane's
#pragma unroll
            for (int j = 7; j >= 0; j--) { run += local[j]; sm.suffix[8 * lane + j] = run; }
            if (lane == 0) sm.suffix[256] = 0;
        }
        __syncthreads();
        const uint32_t rem = sm.remaining;
        __syncthreads();    // every thread has read `remaining` before it changes
        for (int b = threadIdx.x; b < 256; b += blockDim.x) {
            if (sm.suffix[b + 1] < rem && rem <= sm.suffix[b]) {
                sm.prefix = prefix | ((uint64_t)b << shift);
                sm.mask = mask | (255ull << shift);
                sm.remaining = rem - sm.suffix[b + 1];
            }
        }
        __syncthreads();
    }
    return sm.prefix;
}

// Writes the keys >= kth (there are exactly k) to out[0..k).
template <class Keys>
__device__ void gather_at_least(const Keys &key, int64_t m, uint64_t kth, uint64_t *out, SelectSmem &sm)
{
    if (threadIdx.x == 0) sm.count = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        const uint64_t x = key(i);
        if (x != 0 && x >= kth) out[atomicAdd(&sm.count, 1u)] = x;
    }
    __syncthreads();
}

// Batched: blockIdx.y is the query; its scores, candidates, hits and ticket
// sit at y * n, y * (gridDim.x * k), y * hit_stride and y.
__global__ void __launch_bounds__(kTopkThreads)
topk_kernel(const int32_t *scores, int64_t n, int32_t k, uint64_t *cand, int64_t *hit_idx,
            int32_t *hit_score, uint32_t *ticket, int32_t hit_stride)
{
    __shared__ SelectSmem sm;
    __shared__ uint64_t sortbuf[kSortMax];
    __shared__ int is_last;
    scores += (int64_t)blockIdx.y * n;
    cand += (int64_t)blockIdx.y * gridDim.x * k;
    hit_idx += (int64_t)blockIdx.y * hit_stride;
    hit_score += (int64_t)blockIdx.y * hit_stride;
    ticket += blockIdx.y;

    // phase 1: this CTA's slice
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t m = max((int64_t)0, min(n, lo + chunk) - lo);
    uint64_t *mine = cand + (int64_t)blockIdx.x * k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) mine[i] = 0;
    __syncthreads();
    if (m > 0) {
        ScoreKeys keys{scores, lo};
        const uint32_t kk = (uint32_t)min((int64_t)k, m);
        const uint64_t kth = radix_kth(keys, m, kk, sm);
        gather_at_least(keys, m, kth, mine, sm);
    }

    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // phase 2: the k best of all candidates, sorted
    const int64_t mc = (int64_t)gridDim.x * k;
    const uint32_t kk = (uint32_t)min((int64_t)k, n);
    CandKeys ck{cand};
    const uint64_t kth = radix_kth(ck, mc, kk, sm);
    int pow2 = 1;
    while (pow2 < (int)kk) pow2 <<= 1;
    for (int i = threadIdx.x; i < pow2; i += blockDim.x) sortbuf[i] = 0;
    __syncthreads();
    gather_at_least(ck, mc, kth, sortbuf, sm);
    // bitonic sort, descending
    for (int size = 2; size <= pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const uint64_t a = sortbuf[i], b = sortbuf[j];
                    if (desc ? (a < b) : (a > b)) { sortbuf[i] = b; sortbuf[j] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < (int)kk; i += blockDim.x) {
        const uint64_t x = sortbuf[i];
        hit_idx[i] = (int64_t)(0xFFFFFFFFu - (uint32_t)(x & 0xFFFFFFFFu));
        hit_score[i] = (int32_t)((uint32_t)(x >> 32) ^ 0x80000000u);
    }
}

}  // namespace

// Number of pairs scoring at least `threshold` (Sec. IV's threshold score).
__global__ void count_at_least_kernel(const int32_t *scores, int64_t n, int32_t threshold,
                                      unsigned long long *count)
{
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += scores[i] >= threshold;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_count_at_least(const int32_t *scores, int64_t n, int32_t threshold, int64_t *d_count,
                                  int num_sms, cudaStream_t st, int *launches)
{
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
    if (e != cudaSuccess || n <= 0) return e;
    count_at_least_kernel<<<num_sms * 4, 256, 0, st>>>(scores, n, threshold,
                                                       reinterpret_cast<unsigned long long *>(d_count));
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_topk(const Workspace &ws, int64_t n, int32_t k, cudaStream_t st, int *launches)
{
    if (n <= 0 || k <= 0) return cudaSuccess;
    topk_kernel<<<ws.topk_ctas, kTopkThreads, 0, st>>>(ws.scores, n, k, ws.cand, ws.hit_idx, ws.hit_score,
                                                       ws.counters + kTopkTicket, k);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// nhits = min(k, n) best of every query; hit lists are k apart.
cudaError_t launch_topk_batch(const BatchLayout &bl, int64_t n, int32_t k, int32_t nhits, cudaStream_t st,
                              int *launches)
{
    if (n <= 0 || nhits <= 0 || bl.nq <= 0) return cudaSuccess;
    topk_kernel<<<dim3(kTopkCtas, bl.nq), kTopkThreads, 0, st>>>(bl.scores, n, nhits, bl.cand, bl.hit_idx,
                                                                 bl.hit_score, bl.topk_tickets, k);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Word offsets of every query's two profiles (prefix sums, one warp).
__global__ void prof_offsets_kernel(const int64_t *qoffsets, int32_t nq, int64_t *prof_off)
{
    const int lane = threadIdx.x;
    int64_t carry = 0;
    for (int base = 0; base < nq; base += 32) {
        const int q = base + lane;
        const int64_t v = q < nq ? 2 * profile_words((int)(qoffsets[q + 1] - qoffsets[q])) : 0;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (q < nq) prof_off[q] = carry + incl - v;
        carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
}

cudaError_t launch_prof_offsets(const BatchLayout &bl, cudaStream_t st)
{
    prof_offsets_kernel<<<1, 32, 0, st>>>(bl.qoffsets, bl.nq, bl.prof_off);
    return cudaGetLastError();
}

}  // namespace hs
