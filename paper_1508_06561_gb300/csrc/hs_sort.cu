// hs_sort.cu -- the database's scan schedule, built on the device.
//
// The scan visits the database longest first (ties in database order), so
// that the long targets start early and the short ones fill the end of the
// scan.  The order is a stable least-significant-digit radix sort of the
// key (maxlen - length) with 8-bit digits: per pass, every block counts the
// digits of its tile, one scan turns the counts (digit-major, block-minor)
// into each block's first output position per digit, and every block
// scatters its tile in index order -- equal digits keep their relative
// order (ranks within a warp by __match_any_sync, across the block's warps
// by per-warp counts) -- so after the last pass equal lengths stay in
// database order.  Then the lengths in schedule order and their prefix sums
// (the residues before each schedule position, which the batched scan cuts
// into equal chunks).  Prefix sums run in three passes over up to 128
// blocks: block totals, their prefix, each block's values from its offset.
#include <cuda_runtime.h>

#include <algorithm>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr int kSortThreads = 256;       // one thread per digit value
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = 4096;         // elements per block and pass
constexpr int kScanThreads = 1024;

__global__ void order_keys_kernel(const int64_t *offsets, int64_t n, int32_t maxlen, bool by_length,
                                  uint32_t *keys, int32_t *idx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t len = (int32_t)(offsets[i + 1] - offsets[i]);
        keys[i] = by_length ? (uint32_t)(maxlen - len) : 0u;    // ascending key = longest first
        idx[i] = (int32_t)i;
    }
}

// Digit counts of one tile: hist[digit * nblocks + block].
__global__ void __launch_bounds__(kSortThreads) radix_count_kernel(const uint32_t *keys, int64_t n, int shift,
                                                                   uint32_t *hist)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile, t1 = min(n, t0 + kSortTile);
    for (int64_t i = t0 + threadIdx.x; i < t1; i += kSortThreads) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Prefix sums over [lo, hi) by one block, starting from carry0: each thread
// takes kScanItems consecutive values, the block scans the threads' totals
// (warp shuffles, then one warp over the warp totals), and each thread
// walks its own values calling store(i, sum before i, value i).  A thread
// reads all of its values before it stores, so store may overwrite in[i].
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;   // values per block and pass
constexpr int kScanBlocks = 128;                        // blocks of the multi-block form

template <class In, class Sum, class Store>
__device__ __forceinline__ void block_prefix(const In *in, int64_t lo, int64_t hi, Sum carry0, Store store)
{
    __shared__ Sum warp_sum[kScanThreads / 32];
    __shared__ Sum carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = carry0;
    __syncthreads();
    for (int64_t base = lo; base < hi; base += kScanChunk) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kScanItems;
        Sum v[kScanItems];
        Sum t = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            v[k] = i0 + k < hi ? (Sum)in[i0 + k] : (Sum)0;
            t += v[k];
        }
        Sum x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const Sum y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            Sum w = warp_sum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const Sum y = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;                     // inclusive over warps
        }
        __syncthreads();
        Sum run = carry + (warp ? warp_sum[warp - 1] : (Sum)0) + x - t;
        const Sum next_carry = carry + warp_sum[kScanThreads / 32 - 1];
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            if (i0 + k < hi) store(i0 + k, run, v[k]);
            run += v[k];
        }
        __syncthreads();                            // every thread has read carry and warp_sum
        if (threadIdx.x == 0) carry = next_carry;
        __syncthreads();
    }
}

// The multi-block form: block b owns values [b * per, (b + 1) * per).
// Pass 1: each block's total into sums[b + 1] (sums[0] = 0).  Pass 2 (one
// block): sums becomes the inclusive prefix, so sums[b] is the total before
// block b.  Pass 3: each block's prefix sums from sums[b].
template <class In, class Sum>
__global__ void __launch_bounds__(kScanThreads) block_total_kernel(const In *in, int64_t m, int64_t per, Sum *sums)
{
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(m, lo + per);
    __shared__ Sum part[kScanThreads / 32];
    Sum t = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) t += (Sum)in[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        Sum s = 0;
        for (int w = 0; w < kScanThreads / 32; w++) s += part[w];
        sums[blockIdx.x + 1] = s;
        if (blockIdx.x == 0) sums[0] = 0;
    }
}

template <class Sum>
__global__ void __launch_bounds__(kScanThreads) sums_prefix_kernel(Sum *sums, int nb)
{
    block_prefix<Sum, Sum>(sums, 0, nb + 1, (Sum)0, [&](int64_t i, Sum before, Sum v) { sums[i] = before + v; });
}

// In-place exclusive prefix sum of m counts.
__global__ void __launch_bounds__(kScanThreads) exclusive_scan_kernel(uint32_t *a, int64_t m, int64_t per,
                                                                      const uint32_t *sums)
{
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(m, lo + per);
    block_prefix<uint32_t, uint32_t>(a, lo, hi, sums[blockIdx.x],
                                     [&](int64_t i, uint32_t before, uint32_t) { a[i] = before; });
}

// Scatter one tile in index order to its digits' positions (stable).
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint32_t *kin, const int32_t *iin,
                                                                     uint32_t *kout, int32_t *iout, int64_t n,
                                                                     int shift, const uint32_t *first)
{
    __shared__ uint32_t next[256];                  // the next output position of each digit
    __shared__ uint32_t cnt[kSortWarps][256];       // this round's digits per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    next[threadIdx.x] = first[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile, t1 = min(n, t0 + kSortTile);
    for (int64_t r = t0; r < t1; r += kSortThreads) {
        for (int j = threadIdx.x; j < kSortWarps * 256; j += kSortThreads) (&cnt[0][0])[j] = 0u;
        __syncthreads();
        const int64_t i = r + threadIdx.x;
        const bool valid = i < t1;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t d = valid ? (key >> shift) & 255u : 256u;       // 256: no digit of a real key
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));          // earlier lanes with this digit
        if (valid && rank == 0) cnt[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = next[d] + (uint32_t)rank;
            for (int w = 0; w < warp; w++) pos += cnt[w][d];            // earlier warps with this digit
            kout[pos] = key;
            iout[pos] = iin[i];
        }
        __syncthreads();                            // every thread has read next[] and cnt[]
        uint32_t tot = 0;
        for (int w = 0; w < kSortWarps; w++) tot += cnt[w][threadIdx.x];
        next[threadIdx.x] += tot;
        __syncthreads();
    }
}

// Lengths in schedule order.
__global__ void sorted_lengths_kernel(const int64_t *offsets, const int32_t *order, int64_t n, int32_t *len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = order[i];
        len[i] = (int32_t)(offsets[d + 1] - offsets[d]);
    }
}

// cumres[0] = 0, cumres[i + 1] = cumres[i] + len[i].
__global__ void __launch_bounds__(kScanThreads) residue_prefix_kernel(const int32_t *len, int64_t n, int64_t per,
                                                                      const int64_t *sums, int64_t *cumres)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) cumres[0] = 0;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = min(n, lo + per);
    block_prefix<int32_t, int64_t>(len, lo, hi, sums[blockIdx.x],
                                   [&](int64_t i, int64_t before, int64_t v) { cumres[i + 1] = before + v; });
}

// Prefix sums over m values in up to kScanBlocks blocks of whole chunks;
// sums: nb + 1 words of scratch.
static int scan_blocks(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>(kScanBlocks, (m + kScanChunk - 1) / kScanChunk)); }
static int64_t scan_per(int64_t m, int nb) { return ((m + nb - 1) / nb + kScanItems - 1) / kScanItems * kScanItems; }

}  // namespace

// Scratch carve-up: two key buffers, two index buffers and the digit
// counts, each 256-byte aligned.
static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

size_t schedule_scratch_bytes(int64_t n)
{
    const int64_t nb = std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
    const size_t a = (size_t)std::max<int64_t>(n, 1) * 4;
    return 4 * round256(a) + round256((size_t)nb * 256 * 4) + round256(sizeof(int64_t) * (kScanBlocks + 1));
}

cudaError_t build_schedule(const int64_t *d_offsets, int64_t n, int32_t maxlen, bool by_length, int32_t *d_order,
                           int64_t *d_cumres, int32_t *d_sorted_len, void *d_scratch, cudaStream_t st)
{
    const int64_t nb = std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
    const size_t a = (size_t)std::max<int64_t>(n, 1);
    char *p = static_cast<char *>(d_scratch);
    auto take = [&](size_t bytes) { char *q = p; p += round256(bytes); return q; };
    uint32_t *k0 = reinterpret_cast<uint32_t *>(take(a * 4)), *k1 = reinterpret_cast<uint32_t *>(take(a * 4));
    int32_t *i0 = reinterpret_cast<int32_t *>(take(a * 4)), *i1 = reinterpret_cast<int32_t *>(take(a * 4));
    uint32_t *hist = reinterpret_cast<uint32_t *>(take((size_t)nb * 256 * 4));
    void *sums = take(sizeof(int64_t) * (kScanBlocks + 1));
    if (n == 0) return cudaMemsetAsync(d_cumres, 0, sizeof(int64_t), st);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    order_keys_kernel<<<grid, 256, 0, st>>>(d_offsets, n, maxlen, by_length, k0, i0);
    cudaError_t e = cudaGetLastError();
    // passes over the key's significant bits, ping-ponging between the
    // scratch buffers; d_order is written only once the order is complete
    int bits = 0;
    if (by_length)
        while (bits < 32 && (maxlen >> bits) != 0) bits++;
    uint32_t *kin = k0, *kout = k1;
    int32_t *iin = i0, *iout = i1;
    for (int shift = 0; shift < bits && e == cudaSuccess; shift += 8) {
        radix_count_kernel<<<(int)nb, kSortThreads, 0, st>>>(kin, n, shift, hist);
        const int64_t m = nb * 256;
        const int sb = scan_blocks(m);
        const int64_t per = scan_per(m, sb);
        uint32_t *s32 = static_cast<uint32_t *>(sums);
        block_total_kernel<uint32_t, uint32_t><<<sb, kScanThreads, 0, st>>>(hist, m, per, s32);
        sums_prefix_kernel<uint32_t><<<1, kScanThreads, 0, st>>>(s32, sb);
        exclusive_scan_kernel<<<sb, kScanThreads, 0, st>>>(hist, m, per, s32);
        radix_scatter_kernel<<<(int)nb, kSortThreads, 0, st>>>(kin, iin, kout, iout, n, shift, hist);
        e = cudaGetLastError();
        std::swap(kin, kout);
        std::swap(iin, iout);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, iin, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    sorted_lengths_kernel<<<grid, 256, 0, st>>>(d_offsets, d_order, n, d_sorted_len);
    const int sb = scan_blocks(n);
    const int64_t per = scan_per(n, sb);
    int64_t *s64 = static_cast<int64_t *>(sums);
    block_total_kernel<int32_t, int64_t><<<sb, kScanThreads, 0, st>>>(d_sorted_len, n, per, s64);
    sums_prefix_kernel<int64_t><<<1, kScanThreads, 0, st>>>(s64, sb);
    residue_prefix_kernel<<<sb, kScanThreads, 0, st>>>(d_sorted_len, n, per, s64, d_cumres);
    return cudaGetLastError();
}

}  // namespace hs
