// hs_topk.cu -- ranking of the scanned pairs (Sec. IV: results ranked by
// score; read as the k best).  Order: score descending, then database index
// ascending.  Each pair becomes the 64-bit key
//     ((score ^ 0x80000000) << 32) | (0xFFFFFFFF - index)
// so a larger key is a better hit and all keys are distinct.  Every CTA
// selects the k largest keys of its slice: the threshold score comes from
// 12-bit digit histograms of the score above the slice minimum (one pass
// when the slice's scores span less than 4096 values), ties at the threshold
// go to the lowest indices.  The last CTA to finish finds the k-th score of
// all candidates from one histogram of their scores, sorts the candidates at
// or above it in shared memory and writes the ranked (index, score) list;
// for wide score ranges or too many ties it radix-selects over all
// candidates instead.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr int kSortMax = HS_MAX_K;     // bitonic sort buffer (keys)

struct CandKeys {       // candidates written by the other CTAs (0 = empty slot)
    const uint64_t *cand;
    __device__ __forceinline__ uint64_t operator()(int64_t i) const
    {
        // from L2 (their writes are fenced before the ticket), not volatile,
        // so the loads of a pass overlap
        return __ldcg(cand + i);
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

// Bitonic sort of buf[0, pow2), descending (pow2 a power of two).
__device__ void sort_desc(uint64_t *buf, int pow2)
{
    for (int size = 2; size <= pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const uint64_t a = buf[i], b = buf[j];
                    if (desc ? (a < b) : (a > b)) { buf[i] = b; buf[j] = a; }
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kDigitBits = 12;
constexpr int kBins = 1 << kDigitBits;
constexpr int kBinsPerThread = kBins / kTopkThreads;
static_assert(kBins % kTopkThreads == 0, "histogram bins split evenly over the threads");

struct SliceSmem {
    uint32_t umin, umax;
    uint32_t wsum[kTopkThreads / 32];
    uint32_t bin, above, at_bin;
    uint32_t count, ties;
    uint64_t kth;
};

// The histogram bin holding the `remaining`-th largest key: sets ss.bin and
// ss.above (the keys in the bins above it).  Thread t owns bins
// [t * kBinsPerThread, (t + 1) * kBinsPerThread); suffix sums run over the
// threads.  Ends with a barrier.
__device__ void find_bin(const uint32_t *hist, uint32_t remaining, SliceSmem &ss)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kTopkThreads / 32;
    const int b0 = threadIdx.x * kBinsPerThread;
    uint32_t tot = 0u;
#pragma unroll
    for (int j = 0; j < kBinsPerThread; j++) tot += hist[b0 + j];
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_down_sync(0xFFFFFFFFu, incl, o);
        if (lane + o < 32) incl += y;
    }
    if (lane == 0) ss.wsum[warp] = incl;
    __syncthreads();
    uint32_t run = incl - tot;
    for (int w = warp + 1; w < nw; w++) run += ss.wsum[w];
    for (int j = kBinsPerThread - 1; j >= 0; j--) {
        const uint32_t c = hist[b0 + j];
        if (run < remaining && run + c >= remaining) { ss.bin = (uint32_t)(b0 + j); ss.above = run; }
        run += c;
    }
    __syncthreads();
}

// The kk largest keys of the slice [lo, lo + m) of the scores into out[0,
// kk) (any order); returns the smallest of them.  u = score ^ 0x80000000 is
// the score in key order.  Needs blockDim.x == kTopkThreads.
__device__ uint64_t slice_select(const int32_t *scores, int64_t lo, int64_t m, uint32_t kk, uint64_t *out,
                                 uint32_t *hist, SliceSmem &ss)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kTopkThreads / 32;
    // 1. the slice's range of u
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        const uint32_t u = (uint32_t)__ldg(scores + lo + i) ^ 0x80000000u;
        mn = min(mn, u);
        mx = max(mx, u);
    }
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (threadIdx.x == 0) { ss.umin = 0xFFFFFFFFu; ss.umax = 0u; ss.count = 0u; ss.ties = 0u; ss.kth = 0ull; }
    __syncthreads();
    if (lane == 0) { atomicMin(&ss.umin, mn); atomicMax(&ss.umax, mx); }
    __syncthreads();
    const uint32_t umin = ss.umin, range = ss.umax - umin;
    // 2. the k-th key's score: digits of d = u - umin, most significant first
    const int bits = range ? 32 - __clz(range) : 0;
    int shift = bits > 0 ? ((bits - 1) / kDigitBits) * kDigitBits : 0;
    uint32_t prefix = 0u, remaining = kk;
    for (;;) {
        for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        const uint64_t hi_mask = ~0ull << (shift + kDigitBits);     // digits already fixed
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
            const uint32_t d = ((uint32_t)__ldg(scores + lo + i) ^ 0x80000000u) - umin;
            if ((((uint64_t)(d ^ prefix)) & hi_mask) == 0) atomicAdd(&hist[(d >> shift) & (kBins - 1)], 1u);
        }
        __syncthreads();
        find_bin(hist, remaining, ss);
        prefix |= ss.bin << shift;
        remaining -= ss.above;
        __syncthreads();                            // ss.bin is read before the next pass sets it
        if (shift == 0) break;
        shift -= kDigitBits;
    }
    const uint32_t thr = umin + prefix;             // the k-th key's u; `remaining` keys at it are taken
    // 3. every key above thr, and the first `remaining` at thr in index order
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t base = 0; base < m; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint32_t u = i < m ? (uint32_t)__ldg(scores + lo + i) ^ 0x80000000u : 0u;
        const bool tie = i < m && u == thr, above = i < m && u > thr;
        const unsigned tb = __ballot_sync(0xFFFFFFFFu, tie);
        if (lane == 0) ss.wsum[warp] = (uint32_t)__popc(tb);
        __syncthreads();
        uint32_t rank = ss.ties + (uint32_t)__popc(tb & lt_mask);
        for (int w = 0; w < warp; w++) rank += ss.wsum[w];
        const bool take = above || (tie && rank < remaining);
        if (take) {
            const uint64_t key = ((uint64_t)u << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)(lo + i));
            out[atomicAdd(&ss.count, 1u)] = key;
            if (tie && rank == remaining - 1u) ss.kth = key;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0u;
            for (int w = 0; w < nw; w++) t += ss.wsum[w];
            ss.ties += t;
        }
        __syncthreads();
    }
    return ss.kth;
}

// Batched: blockIdx.y is the query; its scores, candidates, hits and ticket
// sit at y * n, y * (gridDim.x * k), y * hit_stride and y.
__global__ void __launch_bounds__(kTopkThreads)
topk_kernel(const int32_t *scores, int64_t n, int32_t k, uint64_t *cand, int64_t *hit_idx,
            int32_t *hit_score, uint32_t *ticket, int32_t hit_stride)
{
    __shared__ SelectSmem sm;
    __shared__ SliceSmem ss;
    __shared__ union {
        uint64_t sortbuf[kSortMax];         // phase 2
        uint32_t hist[kBins];               // phase 1
    } buf;
    uint64_t *sortbuf = buf.sortbuf;
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
    if (m > 0) slice_select(scores, lo, m, (uint32_t)min((int64_t)k, m), mine, buf.hist, ss);

    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // phase 2: the k best of all candidates, sorted.  The candidates' scores
    // span a narrow range: their histogram gives the k-th score, and the
    // candidates at or above it (the k best plus any ties at that score) are
    // sorted in shared memory.  Wide ranges or too many ties: radix select.
    const int64_t mc = (int64_t)gridDim.x * k;
    const uint32_t kk = (uint32_t)min((int64_t)k, n);
    const int lane = threadIdx.x & 31;
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
    for (int64_t i = threadIdx.x; i < mc; i += blockDim.x) {
        const uint64_t x = __ldcg(cand + i);
        if (x != 0) {
            mn = min(mn, (uint32_t)(x >> 32));
            mx = max(mx, (uint32_t)(x >> 32));
        }
    }
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (threadIdx.x == 0) { ss.umin = 0xFFFFFFFFu; ss.umax = 0u; ss.count = 0u; }
    __syncthreads();
    if (lane == 0) { atomicMin(&ss.umin, mn); atomicMax(&ss.umax, mx); }
    __syncthreads();
    const uint32_t umin = ss.umin;
    bool sorted_here = false;
    int pow2 = 1;
    if (ss.umax - umin < (uint32_t)kBins) {
        uint32_t *hist = buf.hist;
        for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < mc; i += blockDim.x) {
            const uint64_t x = __ldcg(cand + i);
            if (x != 0) atomicAdd(&hist[(uint32_t)(x >> 32) - umin], 1u);
        }
        __syncthreads();
        find_bin(hist, kk, ss);
        if (threadIdx.x == 0) ss.at_bin = hist[ss.bin];
        __syncthreads();
        const uint32_t keep = ss.above + ss.at_bin;     // the candidates at or above the k-th score
        if (keep <= (uint32_t)kSortMax) {
            const uint32_t thr = umin + ss.bin;
            while (pow2 < (int)keep) pow2 <<= 1;
            __syncthreads();                            // the histogram (sharing sortbuf's memory) is done
            for (int64_t i = threadIdx.x; i < mc; i += blockDim.x) {
                const uint64_t x = __ldcg(cand + i);
                if (x != 0 && (uint32_t)(x >> 32) >= thr) sortbuf[atomicAdd(&ss.count, 1u)] = x;
            }
            for (int i = (int)keep + threadIdx.x; i < pow2; i += blockDim.x) sortbuf[i] = 0;
            __syncthreads();
            sorted_here = true;
        }
    }
    if (!sorted_here) {
        CandKeys ck{cand};
        const uint64_t kth = radix_kth(ck, mc, kk, sm);
        pow2 = 1;
        while (pow2 < (int)kk) pow2 <<= 1;
        for (int i = threadIdx.x; i < pow2; i += blockDim.x) sortbuf[i] = 0;
        __syncthreads();
        gather_at_least(ck, mc, kth, sortbuf, sm);
    }
    sort_desc(sortbuf, pow2);
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
