// Host run of the batched scan's work loop (batch_items, with the pair loop
// it calls), cut verbatim out of csrc/hs_scan.cu by the test harness into
// hs_pairs_region.inc and hs_batch_region.inc and compiled as plain C++
// against the stub cuda_runtime.h next to this file.  CTAS CTAs of WARPS
// warps run at once (each with its own barrier, staged profile, plan and
// flat-step slots and counters) and take (query, chunk) items from one
// counter, as the persistent launch does.
//
// usage: batch_emu IN OUT
//   IN  (little-endian): int64 n, int64 nres, int32 nq, int32 ctas, int32 warps,
//       int32 nchunk, int32 chunk_step, int32 smem (1: stage each role's
//       profile, length order; 0: read both from memory, database order),
//       int32 pgp, gop, gep, rounds, uint32 lf_q16, sf_q16, minf_q16,
//       int8 M[24*24], uint8 codes[nres], int64 offsets[n+1],
//       int64 qoffsets[nq+1], uint64 seeds[nq], uint8 queries[qoffsets[nq]]
//   OUT int32 scores[nq][n]
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <thread>
#include <vector>

#include "hs_device.cuh"

namespace hs {
#include "hs_pairs_region.inc"
#include "hs_batch_region.inc"
}

using namespace hs;

template <class T> static bool rd(FILE *f, T *p, size_t n = 1) { return n == 0 || fread(p, sizeof(T), n, f) == n; }

template <bool kSmem, bool P16>
static void run(const DbView &db, const BatchScan &bs, const SParams &sp0, int ctas, int warps, int64_t max_words)
{
    struct Cta {
        std::vector<EmuWarp> ws;
        EmuBarrier bar;
        std::vector<uint4> prof;
        std::vector<Plan> plans;
        std::vector<FlatSlots> slots;
        long long item = 0;
        unsigned pos = 0;
    };
    std::vector<Cta> cs(ctas);
    for (auto &c : cs) {
        c.ws = std::vector<EmuWarp>(warps);
        c.bar.count = 32 * warps;
        c.prof.resize((size_t)(max_words / 4 + 1));
        c.plans.resize((size_t)warps * 32);
        c.slots.resize((size_t)warps);
    }
    std::vector<std::thread> th;
    for (int b = 0; b < ctas; b++)
        for (int t = 0; t < 32 * warps; t++)
            th.emplace_back([&, b, t] {
                Cta &c = cs[b];
                emu_warp = &c.ws[t / 32];
                emu_lane = t % 32;
                emu_cta = &c.bar;
                threadIdx.x = (unsigned)t;
                blockIdx.x = (unsigned)b;
                blockDim.x = (unsigned)(32 * warps);
                gridDim.x = (unsigned)ctas;
                batch_items<kSmem, P16>(db, bs, sp0, c.prof.data(), c.plans.data(), c.slots.data(), c.item, c.pos);
            });
    for (auto &x : th) x.join();
}

int main(int argc, char **argv)
{
    if (argc != 3) { fprintf(stderr, "usage: batch_emu IN OUT\n"); return 2; }
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n, nres;
    int32_t nq, ctas, warps, nchunk, chunk_step, smem, pgp, gop, gep, rounds;
    uint32_t lf, sf, minf;
    int8_t M[kNSym * kNSym];
    bool ok = rd(f, &n) && rd(f, &nres) && rd(f, &nq) && rd(f, &ctas) && rd(f, &warps) && rd(f, &nchunk) &&
              rd(f, &chunk_step) && rd(f, &smem) && rd(f, &pgp) && rd(f, &gop) && rd(f, &gep) && rd(f, &rounds) &&
              rd(f, &lf) && rd(f, &sf) && rd(f, &minf) && rd(f, M, sizeof(M));
    std::vector<uint8_t> codes((size_t)nres + kCodesPad, 0);
    std::vector<int64_t> offsets((size_t)n + 1), qoffsets((size_t)nq + 1);
    std::vector<uint64_t> seeds((size_t)nq);
    ok = ok && rd(f, codes.data(), (size_t)nres) && rd(f, offsets.data(), (size_t)n + 1) &&
         rd(f, qoffsets.data(), (size_t)nq + 1) && rd(f, seeds.data(), (size_t)nq);
    std::vector<uint8_t> queries((size_t)std::max<int64_t>(qoffsets[nq], 1));
    ok = ok && rd(f, queries.data(), (size_t)qoffsets[nq]);
    fclose(f);
    if (!ok) { fprintf(stderr, "short input\n"); return 2; }

    // schedule: longest first (length order) or database order
    std::vector<int32_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    auto len = [&](int32_t d) { return offsets[d + 1] - offsets[d]; };
    if (smem) std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return len(a) > len(b); });
    int64_t long_end = 0;
    if (smem) while (long_end < n && len(order[long_end]) >= kLongLen) long_end++;
    // scoring parameters (the per-query length and seed are set by the loop)
    int lo = 127, hi = -128;
    for (int i = 0; i < kNSym * kNSym; i++) { lo = std::min<int>(lo, M[i]); hi = std::max<int>(hi, M[i]); }
    int32_t max_qlen = 0;
    for (int q = 0; q < nq; q++) max_qlen = std::max<int32_t>(max_qlen, (int32_t)(qoffsets[q + 1] - qoffsets[q]));
    SParams sp = {};
    sp.flat_min_chunks = kFlatMinChunks;
    sp.flat_max_iters = kFlatMaxIters;
    sp.bias = -lo;
    const int range = hi - lo;
    sp.flush = range == 0 ? 255 : std::max(1, 255 / range);
    sp.pgp = pgp; sp.gop = gop; sp.gep = gep; sp.rounds = rounds;
    sp.lf_q16 = lf; sp.sf_q16 = sf; sp.minf_q16 = minf;
    sp.min_score = INT_MIN;
    sp.mode = HS_MODE_DB;
    sp.pair16 = (int64_t)range * (max_qlen + 3) <= 65535;
    // both role profiles of every query, back to back
    std::vector<int64_t> prof_off((size_t)nq);
    int64_t total = 0, max_words = 0;
    for (int q = 0; q < nq; q++) {
        prof_off[q] = total;
        const int64_t w = profile_words((int)(qoffsets[q + 1] - qoffsets[q]));
        total += 2 * w;
        max_words = std::max(max_words, w);
    }
    std::vector<uint32_t> prof((size_t)total);
    for (int q = 0; q < nq; q++) {
        const int ql = (int)(qoffsets[q + 1] - qoffsets[q]);
        const uint8_t *qs = queries.data() + qoffsets[q];
        const int R = profile_stride(ql);
        const int64_t w = profile_words(ql);
        for (int a = 0; a < kNSym; a++)
            for (int s = 0; s < R; s++) {
                prof[prof_off[q] + (size_t)a * R + s] = profile_word_value(qs, ql, true, M, sp.bias, a, s);
                prof[prof_off[q] + w + (size_t)a * R + s] = profile_word_value(qs, ql, false, M, sp.bias, a, s);
            }
    }
    // chunks: equal numbers of positions (any split gives the same scores)
    std::vector<int64_t> bounds((size_t)nchunk + 1);
    for (int c = 0; c <= nchunk; c++) bounds[c] = n * c / nchunk;
    std::vector<int32_t> qlist((size_t)nq);
    std::iota(qlist.begin(), qlist.end(), 0);
    const unsigned qcount = (unsigned)nq;
    unsigned item_ctr = 0;
    std::vector<int32_t> scores((size_t)nq * n, INT32_MIN + 1);
    BatchScan bs = {};
    bs.nq = nq;
    bs.nchunk = nchunk;
    bs.qlist = qlist.data();
    bs.qcount = &qcount;
    bs.qoffsets = qoffsets.data();
    bs.seeds = seeds.data();
    bs.prof_off = prof_off.data();
    bs.prof = prof.data();
    bs.bounds = bounds.data();
    bs.long_end = long_end;
    bs.scores = scores.data();
    bs.item_ctr = &item_ctr;
    bs.smem_words = smem ? max_words : 0;
    bs.chunk_step = chunk_step;
    const DbView db = {codes.data(), offsets.data(), order.data(), n};
    if (smem) {
        if (sp.pair16) run<true, true>(db, bs, sp, ctas, warps, max_words);
        else run<true, false>(db, bs, sp, ctas, warps, max_words);
    } else {
        if (sp.pair16) run<false, true>(db, bs, sp, ctas, warps, max_words);
        else run<false, false>(db, bs, sp, ctas, warps, max_words);
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(scores.data(), sizeof(int32_t), scores.size(), o);
    fclose(o);
    return 0;
}
