// Host run of the top-k kernel (csrc/hs_topk.cu, cut out verbatim by the
// test harness into hs_topk_region.inc), compiled as plain C++ against the
// stub cuda_runtime.h next to this file: each CTA is kTopkThreads threads
// (warps in lockstep, a CTA barrier for __syncthreads), and the CTAs run one
// after another, so the last one to take the ticket merges, as on the GPU.
//
// usage: topk_emu IN OUT
//   IN  (little-endian): int64 n, int32 k, int32 ctas, int32 scores[n]
//   OUT int64 hit_idx[min(k, n)], int32 hit_score[min(k, n)]
#include <algorithm>
#include <cstdio>
#include <thread>
#include <vector>

#include "hs_internal.h"

namespace hs {
#include "hs_topk_region.inc"
}

using namespace hs;

int main(int argc, char **argv)
{
    if (argc != 3) { fprintf(stderr, "usage: topk_emu IN OUT\n"); return 2; }
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n;
    int32_t k, ctas;
    bool ok = fread(&n, 8, 1, f) == 1 && fread(&k, 4, 1, f) == 1 && fread(&ctas, 4, 1, f) == 1;
    std::vector<int32_t> scores((size_t)std::max<int64_t>(n, 1));
    ok = ok && (n == 0 || fread(scores.data(), 4, (size_t)n, f) == (size_t)n);
    fclose(f);
    if (!ok || k < 1 || ctas < 1) { fprintf(stderr, "bad input\n"); return 2; }

    std::vector<uint64_t> cand((size_t)ctas * k, 0xDEADBEEFull);    // the kernel clears its own slots
    std::vector<int64_t> hit_idx((size_t)k, -1);
    std::vector<int32_t> hit_score((size_t)k, 0);
    uint32_t ticket = 0;
    constexpr int kWarps = kTopkThreads / 32;
    for (int c = 0; c < ctas; c++) {
        std::vector<EmuWarp> ws(kWarps);
        EmuBarrier cta;
        cta.count = kTopkThreads;
        std::vector<std::thread> th;
        for (int t = 0; t < kTopkThreads; t++)
            th.emplace_back([&, c, t] {
                emu_warp = &ws[t / 32];
                emu_lane = t % 32;
                emu_cta = &cta;
                threadIdx.x = (unsigned)t;
                blockIdx.x = (unsigned)c;
                blockIdx.y = 0;
                blockDim.x = kTopkThreads;
                gridDim.x = (unsigned)ctas;
                gridDim.y = 1;
                topk_kernel(scores.data(), n, k, cand.data(), hit_idx.data(), hit_score.data(), &ticket, k);
            });
        for (auto &x : th) x.join();
    }
    const int64_t nh = std::min<int64_t>(k, n);
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(hit_idx.data(), 8, (size_t)nh, o);
    fwrite(hit_score.data(), 4, (size_t)nh, o);
    fclose(o);
    return 0;
}
