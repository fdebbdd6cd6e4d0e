// Host run of the scan's step sharing (share_step / help_out, cut from
// csrc/hs_scan.cu into hs_pairs_region.inc like the pair loop): one owner
// warp publishes a flat step of a random window and takes passes of it.
//
//   ok    -- a second warp, out of pairs, helps; the step's key must equal
//            the maximum of its units' keys computed one by one, both warps
//            must leave and the status must stay HS_OK;
//   stuck -- a stand-in for a helper claims one pass and never finishes it;
//            the owner must give up after its wait limit, record
//            HS_ETIMEOUT and return.
//
// usage: help_emu ok|stuck SEED   (prints "key K want W status S ms T claimed C")
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "hs_device.cuh"

namespace hs {
#include "hs_pairs_region.inc"
}

using namespace hs;

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    const std::string how = argv[1];
    std::mt19937_64 rng(atoi(argv[2]));
    int8_t M[kNSym * kNSym];
    for (int a = 0; a < kNSym; a++)
        for (int b = 0; b <= a; b++) M[a * kNSym + b] = M[b * kNSym + a] = (int8_t)((int)(rng() % 16) - 4);
    const int qlen = 40, tlen = 3000;
    std::vector<uint8_t> q(qlen), t((size_t)tlen + kCodesPad, 0);
    for (auto &c : q) c = (uint8_t)(rng() % 24);
    for (int i = 0; i < tlen; i++) t[i] = (uint8_t)(rng() % 24);
    SParams sp = {};
    sp.bias = 4;
    sp.flush = 255 / 15;
    sp.qlen = qlen;
    const int R = profile_stride(qlen);
    const int64_t words = profile_words(qlen);
    std::vector<uint32_t> prof_rev((size_t)words), prof_fwd((size_t)words);
    for (int a = 0; a < kNSym; a++)
        for (int s = 0; s < R; s++) {
            prof_rev[(size_t)a * R + s] = profile_word_value(q.data(), qlen, true, M, sp.bias, a, s);
            prof_fwd[(size_t)a * R + s] = profile_word_value(q.data(), qlen, false, M, sp.bias, a, s);
        }
    QueryCtx qc = {prof_rev.data(), prof_fwd.data(), nullptr, nullptr};
    Plan g = {t.data(), 100, 5, 2000, 20, 1, 0, 0, 0};
    const unsigned units = (unsigned)((g.ls - g.ss + 4) >> 2);

    std::vector<FlatSlots> slots(2);
    std::vector<HelpBoard> boards(2);
    slots[0].desc[0] = flat_desc(g, qlen);
    unsigned live = 2;
    int32_t status = 0;
    const Help help = {slots.data(), boards.data(), 2, &live, &status};

    uint32_t want = 0;
    for (unsigned u = 0; u < units; u++)
        want = std::max(want, desc_key(qc.prof_rev, qc.prof_fwd, R, slots[0].desc[0], 4 * (int)u, sp.flush));

    std::vector<EmuWarp> ws(2);
    std::vector<std::thread> th;
    std::atomic<unsigned> claimed{0};
    const auto t0 = std::chrono::steady_clock::now();
    for (int lane = 0; lane < 32; lane++)
        th.emplace_back([&, lane] {
            emu_warp = &ws[0];
            emu_lane = lane;
            share_step(&help, &slots[0], units, qc, R, sp, lane);
            if (how == "ok") help_out(&help, qc, R, sp, lane);       // the owner, out of pairs too
        });
    if (how == "ok") {
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, lane] {
                emu_warp = &ws[1];
                emu_lane = lane;
                help_out(&help, qc, R, sp, lane);
            });
    } else {
        // take one pass as soon as the step is published, and never finish it
        th.emplace_back([&] {
            for (;;) {
                const unsigned long long c = __atomic_load_n(&boards[0].claim, __ATOMIC_ACQUIRE);
                if ((unsigned)(c >> 32) != 0) break;
                std::this_thread::yield();
            }
            const unsigned long long x = atomicAdd(&boards[0].claim, 32ull);
            if ((unsigned)x < (unsigned)(x >> 32)) claimed = 1;
        });
    }
    for (auto &x : th) x.join();
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    printf("key %u want %u status %d ms %.0f claimed %u live %u\n", slots[0].key[0], want, status, ms,
           claimed.load(), live);
    return 0;
}
