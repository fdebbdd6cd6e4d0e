// Host run of the database-load kernels (csrc/hs_sort.cu's device code, cut
// out into hs_sort_region.inc as it stands) against the stub
// cuda_runtime.h: every CTA of a launch runs in turn as real threads, 32 to
// a lockstep warp, with a CTA barrier.
//
//   sort IN OUT -- IN: int64 n, int64 offsets[n + 1].  The launch sequence of
//                  build_schedule (order keys; per 8-bit digit: counts, the
//                  three-pass prefix of the counts, stable scatter; lengths
//                  in order; three-pass residue prefix).  OUT: int32
//                  order[n], int64 cumres[n + 1].
//   scan IN OUT -- IN: int64 m, uint32 a[m].  The three-pass exclusive
//                  prefix alone.  OUT: uint32 prefix[m].
#include <cstdio>
#include <cstdlib>
#include <string>
#include <thread>
#include <vector>

#include "cuda_runtime.h"
#include "hs_internal.h"

namespace hs {
namespace {
#include "hs_sort_region.inc"
}
}  // namespace hs

using namespace hs;

// every CTA of a grid in turn, `threads` host threads each
template <class F> static void launch(int grid, int threads, F body)
{
    for (int b = 0; b < grid; b++) {
        std::vector<EmuWarp> ws((size_t)threads / 32);
        EmuBarrier cta;
        cta.count = threads;
        std::vector<std::thread> th;
        for (int t = 0; t < threads; t++)
            th.emplace_back([&, b, t] {
                emu_warp = &ws[(size_t)t / 32];
                emu_lane = t & 31;
                emu_cta = &cta;
                threadIdx.x = (unsigned)t;
                blockIdx.x = (unsigned)b;
                blockDim.x = (unsigned)threads;
                gridDim.x = (unsigned)grid;
                body();
            });
        for (auto &x : th) x.join();
    }
}

int main(int argc, char **argv)
{
    if (argc != 4) { fprintf(stderr, "usage: sort_emu sort|scan IN OUT\n"); return 2; }
    const std::string how = argv[1];
    FILE *f = fopen(argv[2], "rb");
    if (!f) return 2;
    int64_t n = 0;
    if (fread(&n, 8, 1, f) != 1) return 2;
    if (how == "scan") {
        std::vector<uint32_t> a((size_t)n);
        if (fread(a.data(), 4, (size_t)n, f) != (size_t)n) return 2;
        fclose(f);
        std::vector<uint32_t> sums(kScanBlocks + 1);
        const int sb = scan_blocks(n);
        const int64_t per = scan_per(n, sb);
        launch(sb, kScanThreads, [&] { block_total_kernel<uint32_t, uint32_t>(a.data(), n, per, sums.data()); });
        launch(1, kScanThreads, [&] { sums_prefix_kernel<uint32_t>(sums.data(), sb); });
        launch(sb, kScanThreads, [&] { exclusive_scan_kernel(a.data(), n, per, sums.data()); });
        FILE *o = fopen(argv[3], "wb");
        fwrite(a.data(), 4, a.size(), o);
        fclose(o);
        return 0;
    }
    std::vector<int64_t> offsets((size_t)n + 1);
    if (fread(offsets.data(), 8, (size_t)n + 1, f) != (size_t)n + 1) return 2;
    fclose(f);
    int32_t maxlen = 0;
    for (int64_t i = 0; i < n; i++) maxlen = std::max<int32_t>(maxlen, (int32_t)(offsets[i + 1] - offsets[i]));
    const int64_t nb = std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
    std::vector<uint32_t> k0((size_t)n), k1((size_t)n), hist((size_t)nb * 256);
    std::vector<int32_t> i0((size_t)n), i1((size_t)n), len((size_t)n);
    std::vector<int64_t> cumres((size_t)n + 1);
    std::vector<int64_t> sums(kScanBlocks + 1);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    launch(grid, 256, [&] { order_keys_kernel(offsets.data(), n, maxlen, true, k0.data(), i0.data()); });
    int bits = 0;
    while (bits < 32 && (maxlen >> bits) != 0) bits++;
    uint32_t *kin = k0.data(), *kout = k1.data();
    int32_t *iin = i0.data(), *iout = i1.data();
    for (int shift = 0; shift < bits; shift += 8) {
        launch((int)nb, kSortThreads, [&] { radix_count_kernel(kin, n, shift, hist.data()); });
        const int64_t m = nb * 256;
        const int sb = scan_blocks(m);
        const int64_t per = scan_per(m, sb);
        uint32_t *s32 = reinterpret_cast<uint32_t *>(sums.data());
        launch(sb, kScanThreads, [&] { block_total_kernel<uint32_t, uint32_t>(hist.data(), m, per, s32); });
        launch(1, kScanThreads, [&] { sums_prefix_kernel<uint32_t>(s32, sb); });
        launch(sb, kScanThreads, [&] { exclusive_scan_kernel(hist.data(), m, per, s32); });
        launch((int)nb, kSortThreads, [&] { radix_scatter_kernel(kin, iin, kout, iout, n, shift, hist.data()); });
        std::swap(kin, kout);
        std::swap(iin, iout);
    }
    launch(grid, 256, [&] { sorted_lengths_kernel(offsets.data(), iin, n, len.data()); });
    const int sb = scan_blocks(n);
    const int64_t per = scan_per(n, sb);
    launch(sb, kScanThreads, [&] { block_total_kernel<int32_t, int64_t>(len.data(), n, per, sums.data()); });
    launch(1, kScanThreads, [&] { sums_prefix_kernel<int64_t>(sums.data(), sb); });
    launch(sb, kScanThreads, [&] { residue_prefix_kernel(len.data(), n, per, sums.data(), cumres.data()); });
    FILE *o = fopen(argv[3], "wb");
    fwrite(iin, 4, (size_t)n, o);
    fwrite(cumres.data(), 8, cumres.size(), o);
    fclose(o);
    return 0;
}
