// Host run of the scan's whole pair loop (run_pairs, the code every scan
// kernel's warps execute), compiled as plain C++ against the stub
// cuda_runtime.h next to this file: each warp is 32 threads in lockstep,
// shared-memory slots are host arrays, the queue counter is a host atomic.
// The test harness extracts run_pairs and its helpers from csrc/hs_scan.cu
// into hs_pairs_region.inc (so the code run here is the kernel source
// itself) and compares the per-pair scores and cell counts this writes with
// the oracle's.
//
// With a third argument "whole", each warp instead takes whole
// pairs from the queue and scores them with align_pair -- the one-warp-per-
// pair path of the full-slide scan, the replay and hs_get_alignment -- in
// the mode the input names.  With "cta", one CTA of `warps` warps takes
// each pair and every step is scanned by all its warps (align_round_cta,
// the replay's path for one-round searches).  With "ops" or "ops_cta" the
// pairs are replayed as the replay kernel does it -- best round found, then
// that round run again writing run-length ops, by one warp or (one round)
// by one CTA -- and OUT gets, per pair in database order, int32 score,
// int32 ops count, int32 span[4] (q begin, q end, t begin, t end) and the
// ops.
//
// With "lanes" (full-slide mode, 16-bit pair sums), every lane holds one
// (position, round) item (run_full_pairs).
//
// usage: pairs_emu IN OUT [whole|lanes|cta|ops|ops_cta]
//   IN  (little-endian): int64 n, int64 nres, int32 qlen, int32 warps,
//       int32 pgp, gop, gep, rounds, mode, uint32 lf_q16, sf_q16, minf_q16,
//       uint64 seed, int64 index_base, int8 M[24*24] (M[query][target]),
//       uint8 codes[nres], int64 offsets[n+1], uint8 query[qlen]
//   OUT int32 scores[n], int64 cells[n], int32 pair16, int64 long_end
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "hs_device.cuh"

namespace hs {
#include "hs_pairs_region.inc"
}

using namespace hs;

template <class T> static bool rd(FILE *f, T *p, size_t n = 1) { return fread(p, sizeof(T), n, f) == n; }

// the warps form one CTA of the wide kernel: idle warps help with the
// others' large lone steps (sp.help_min_units; env HS_EMU_HELP_MIN)
static int32_t g_status = 0;
template <bool P16>
static void run(const DbView &db, const SParams &sp, const QueryCtx &qc, const PosQueue &pq, int warps)
{
    std::vector<EmuWarp> ws(warps);
    std::vector<Plan> plans((size_t)warps * 32);
    std::vector<FlatSlots> slots(warps);
    std::vector<HelpBoard> boards(warps);
    unsigned live = (unsigned)warps;
    const Help help = {slots.data(), boards.data(), warps, &live, &g_status};
    std::vector<std::thread> th;
    for (int w = 0; w < warps; w++)
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, w, lane] {
                emu_warp = &ws[w];
                emu_lane = lane;
                run_pairs<P16, true>(db, sp, qc, pq, plans.data() + 32 * w, &slots[w], lane, &help);
            });
    for (auto &t : th) t.join();
    // 32-bit sums share no step, so their warps never leave through the helper loop
    if ((P16 && live != 0) || g_status != 0) { fprintf(stderr, "help: live %u status %d\n", live, g_status); exit(3); }
}

// the full-slide scan's (position, round) items, by the kernel's own loop
static void run_full(const DbView &db, const SParams &sp, const QueryCtx &qc, const PosQueue &pq, int warps)
{
    std::fill(qc.scores, qc.scores + db.n, INT_MIN);
    std::fill(qc.cells, qc.cells + db.n, 0);
    unsigned long long ctr = 0;
    const FullQueue fq = {pq.begin, pq.end, &ctr, qc.prof_rev, qc.prof_fwd, pq.begin};
    std::vector<EmuWarp> ws(warps);
    std::vector<std::thread> th;
    for (int w = 0; w < warps; w++)
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, w, lane] {
                emu_warp = &ws[w];
                emu_lane = lane;
                run_full_items(db, sp, fq, qc.scores, qc.cells, lane);
            });
    for (auto &t : th) t.join();
}

// the full-slide scan's lane-owned form: every lane holds a (position,
// round) item, the warp's flat steps dealt as units (run_full_pairs)
static void run_full_lanes(const DbView &db, const SParams &sp, const QueryCtx &qc, const PosQueue &pq, int warps)
{
    std::fill(qc.scores, qc.scores + db.n, INT_MIN);
    std::fill(qc.cells, qc.cells + db.n, 0);
    unsigned long long ctr = 0;
    const FullQueue fq = {pq.begin, pq.end, &ctr, qc.prof_rev, qc.prof_fwd, pq.long_end};
    std::vector<EmuWarp> ws(warps);
    std::vector<Plan> plans((size_t)warps * 32);
    std::vector<FlatSlots> slots(warps);
    std::vector<std::thread> th;
    for (int w = 0; w < warps; w++)
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, w, lane] {
                emu_warp = &ws[w];
                emu_lane = lane;
                run_full_pairs(db, sp, qc, fq, pq.lanes, &slots[w], plans.data() + 32 * w, lane);
            });
    for (auto &t : th) t.join();
}

// one pair per warp at a time (align_pair: the path of the one-warp replay
// and hs_get_alignment)
static void run_whole(const DbView &db, const SParams &sp, const QueryCtx &qc, const PosQueue &pq, int warps)
{
    if (sp.mode == HS_MODE_FULL) {
        run_full(db, sp, qc, pq, warps);
        return;
    }
    std::vector<EmuWarp> ws(warps);
    std::vector<std::thread> th;
    for (int w = 0; w < warps; w++)
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, w, lane] {
                emu_warp = &ws[w];
                emu_lane = lane;
                for (;;) {
                    long long pos = 0;
                    if (lane == 0) pos = (long long)pq.begin + (long long)atomicAdd(pq.ctr, 1u);
                    pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
                    if (pos >= pq.end) break;
                    const int64_t d = db.order[pos];
                    PairCtx c;
                    c.t = db.codes + db.offsets[d];
                    c.tlen = (int32_t)(db.offsets[d + 1] - db.offsets[d]);
                    c.qlen = sp.qlen;
                    c.qsmall = c.tlen >= sp.qlen;
                    c.prof = c.qsmall ? qc.prof_rev : qc.prof_fwd;
                    c.S = profile_stride(sp.qlen);
                    int64_t cells = 0;
                    const int32_t sc = align_pair(c, sp, (uint64_t)d, lane, cells, nullptr);
                    if (lane == 0) {
                        qc.scores[d] = sc;
                        qc.cells[d] = cells;
                    }
                }
            });
    for (auto &t : th) t.join();
}

// one CTA: each pair's steps split over all its warps, rounds in turn
static void run_cta(const DbView &db, const SParams &sp, const QueryCtx &qc, const PosQueue &pq, int warps)
{
    std::vector<EmuWarp> ws(warps);
    EmuBarrier cta;
    cta.count = 32 * warps;
    std::vector<int2> red(warps);
    long long claim = 0;
    std::vector<std::thread> th;
    for (int w = 0; w < warps; w++)
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, w, lane] {
                emu_warp = &ws[w];
                emu_lane = lane;
                emu_cta = &cta;
                const bool lead = w == 0 && lane == 0;
                for (;;) {
                    if (lead) claim = (long long)pq.begin + (long long)atomicAdd(pq.ctr, 1u);
                    __syncthreads();
                    const long long pos = claim;
                    __syncthreads();
                    if (pos >= pq.end) break;
                    const int64_t d = db.order[pos];
                    PairCtx c;
                    c.t = db.codes + db.offsets[d];
                    c.tlen = (int32_t)(db.offsets[d + 1] - db.offsets[d]);
                    c.qlen = sp.qlen;
                    c.qsmall = c.tlen >= sp.qlen;
                    c.prof = c.qsmall ? qc.prof_rev : qc.prof_fwd;
                    c.S = profile_stride(sp.qlen);
                    int64_t cells = 0;
                    int32_t best = INT_MIN;
                    for (int r = 0; r < sp.rounds; r++) {
                        const int32_t sc = align_round_cta<false>(c, sp, (uint64_t)d, r, lane, w, warps, red.data(),
                                                                  cells, nullptr, nullptr);
                        if (sc > best) best = sc;
                    }
                    if (lead) {
                        qc.scores[d] = best;
                        qc.cells[d] = cells;
                    }
                }
            });
    for (auto &t : th) t.join();
}

// the replay's emission, one warp (cta = false) or one CTA per pair
struct Replayed {
    int32_t score = 0;
    Span span = {-1, -1, -1, -1};
    std::vector<uint32_t> ops;
};
static void run_replay(const DbView &db, const SParams &sp, const QueryCtx &qc, const PosQueue &pq, int warps,
                       bool cta_mode, std::vector<Replayed> &out)
{
    const int nw = cta_mode ? warps : 1;         // warps per pair
    const int groups = cta_mode ? 1 : warps;
    std::vector<EmuWarp> ws(warps);
    std::vector<EmuBarrier> bars(groups);
    for (auto &b : bars) b.count = 32 * nw;
    std::vector<int2> red(warps);
    std::vector<long long> claim(groups);
    std::vector<std::thread> th;
    for (int w = 0; w < warps; w++)
        for (int lane = 0; lane < 32; lane++)
            th.emplace_back([&, w, lane] {
                const int g = cta_mode ? 0 : w, wi = cta_mode ? w : 0;
                emu_warp = &ws[w];
                emu_lane = lane;
                emu_cta = &bars[g];
                const bool lead = wi == 0 && lane == 0;
                for (;;) {
                    if (lead) claim[g] = (long long)pq.begin + (long long)atomicAdd(pq.ctr, 1u);
                    __syncthreads();
                    const long long pos = claim[g];
                    __syncthreads();
                    if (pos >= pq.end) break;
                    const int64_t d = db.order[pos];
                    PairCtx c;
                    c.t = db.codes + db.offsets[d];
                    c.tlen = (int32_t)(db.offsets[d + 1] - db.offsets[d]);
                    c.qlen = sp.qlen;
                    c.qsmall = c.tlen >= sp.qlen;
                    c.prof = c.qsmall ? qc.prof_rev : qc.prof_fwd;
                    c.S = profile_stride(sp.qlen);
                    std::vector<uint32_t> buf((size_t)c.tlen + sp.qlen + 8);
                    OpWriter ow;
                    ow.init(buf.data(), (int64_t)buf.size());
                    Span span = {-1, -1, -1, -1};
                    int64_t cells = 0;
                    int32_t sc;
                    if (cta_mode) {
                        sc = align_round_cta<true>(c, sp, (uint64_t)d, 0, lane, wi, nw, red.data(), cells, &ow, &span);
                    } else {
                        int br = 0;
                        align_pair(c, sp, (uint64_t)d, lane, cells, &br);
                        sc = sp.mode == HS_MODE_FULL
                                 ? align_round_full<true>(c, sp, (uint64_t)d, br, lane, cells, &ow, &span)
                                 : align_round<true>(c, sp, (uint64_t)d, br, lane, cells, &ow, &span);
                    }
                    if (lead) {
                        Replayed &r = out[d];
                        r.score = sc;
                        r.span = span;
                        r.ops.assign(buf.begin(), buf.begin() + std::min<int64_t>(ow.n, (int64_t)buf.size()));
                    }
                }
            });
    for (auto &t : th) t.join();
}

int main(int argc, char **argv)
{
    if (argc != 3 && argc != 4) { fprintf(stderr, "usage: pairs_emu IN OUT [whole|lanes|cta|ops|ops_cta]\n"); return 2; }
    const std::string how = argc == 4 ? argv[3] : "";
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t n, nres, index_base;
    int32_t qlen, warps, pgp, gop, gep, rounds, mode;
    uint32_t lf, sf, minf;
    uint64_t seed;
    int8_t M[kNSym * kNSym];
    bool ok = rd(f, &n) && rd(f, &nres) && rd(f, &qlen) && rd(f, &warps) && rd(f, &pgp) && rd(f, &gop) &&
              rd(f, &gep) && rd(f, &rounds) && rd(f, &mode) && rd(f, &lf) && rd(f, &sf) && rd(f, &minf) &&
              rd(f, &seed) && rd(f, &index_base) && rd(f, M, sizeof(M));
    std::vector<uint8_t> codes((size_t)nres + kCodesPad, 0);
    std::vector<int64_t> offsets((size_t)n + 1);
    std::vector<uint8_t> q((size_t)qlen);
    ok = ok && rd(f, codes.data(), (size_t)nres) && rd(f, offsets.data(), (size_t)n + 1) &&
         rd(f, q.data(), (size_t)qlen);
    fclose(f);
    if (!ok) { fprintf(stderr, "short input\n"); return 2; }

    // the library's host setup: length order (longest first), matrix bias,
    // byte-lane flush interval, accumulator form, both role profiles
    std::vector<int32_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    auto len = [&](int32_t d) { return offsets[d + 1] - offsets[d]; };
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return len(a) > len(b); });
    int64_t long_end = 0;
    while (long_end < n && len(order[long_end]) >= kLongLen) long_end++;
    int lo = 127, hi = -128;
    for (int i = 0; i < kNSym * kNSym; i++) { lo = std::min<int>(lo, M[i]); hi = std::max<int>(hi, M[i]); }
    SParams sp = {};
    // the flat-list thresholds (a batched search's tuning may change them)
    const char *fmin = getenv("HS_EMU_FLAT_MIN_CHUNKS"), *fmax = getenv("HS_EMU_FLAT_MAX_ITERS");
    sp.flat_min_chunks = fmin ? atoi(fmin) : kFlatMinChunks;
    sp.flat_max_iters = fmax ? atoi(fmax) : kFlatMaxIters;
    const char *hmin = getenv("HS_EMU_HELP_MIN");
    sp.help_min_units = hmin ? atoi(hmin) : kHelpMinUnits;
    sp.bias = -lo;
    const int range = hi - lo;
    sp.flush = range == 0 ? 255 : std::max(1, 255 / range);
    sp.pgp = pgp; sp.gop = gop; sp.gep = gep; sp.rounds = rounds;
    sp.lf_q16 = lf; sp.sf_q16 = sf; sp.minf_q16 = minf;
    sp.qlen = qlen;
    sp.seed = seed;
    sp.index_base = index_base;
    sp.min_score = INT_MIN;
    sp.mode = mode;
    sp.pair16 = (int64_t)range * (qlen + 3) <= 65535;
    const int R = profile_stride(qlen);
    const int64_t words = profile_words(qlen);
    std::vector<uint32_t> prof_rev((size_t)words), prof_fwd((size_t)words);
    for (int a = 0; a < kNSym; a++)
        for (int s = 0; s < R; s++) {
            prof_rev[(size_t)a * R + s] = profile_word_value(q.data(), qlen, true, M, sp.bias, a, s);
            prof_fwd[(size_t)a * R + s] = profile_word_value(q.data(), qlen, false, M, sp.bias, a, s);
        }

    std::vector<int32_t> scores((size_t)n, INT32_MIN + 1);
    std::vector<int64_t> cells((size_t)n, -1);
    unsigned ctr = 0;
    const DbView db = {codes.data(), offsets.data(), order.data(), n};
    QueryCtx qc;
    qc.prof_rev = prof_rev.data();
    qc.prof_fwd = prof_fwd.data();
    qc.scores = scores.data();
    qc.cells = cells.data();
    // lanes a warp fills (the library spreads a small database thin)
    const char *lanes_env = getenv("HS_EMU_LANES");
    const int lanes = lanes_env ? atoi(lanes_env) : 32;
    const PosQueue pq = {0, long_end, n, &ctr, lanes >= 32 ? 0xFFFFFFFFu : (1u << lanes) - 1u};
    if (how == "ops" || how == "ops_cta") {
        std::vector<Replayed> rep((size_t)n);
        run_replay(db, sp, qc, pq, warps, how == "ops_cta", rep);
        FILE *o = fopen(argv[2], "wb");
        if (!o) return 2;
        for (const Replayed &r : rep) {
            const int32_t hdr[6] = {r.score, (int32_t)r.ops.size(), r.span.qb, r.span.qe, r.span.tb, r.span.te};
            fwrite(hdr, sizeof(int32_t), 6, o);
            fwrite(r.ops.data(), sizeof(uint32_t), r.ops.size(), o);
        }
        fclose(o);
        return 0;
    }
    if (how == "whole") run_whole(db, sp, qc, pq, warps);
    else if (how == "lanes") run_full_lanes(db, sp, qc, pq, warps);
    else if (how == "cta") run_cta(db, sp, qc, pq, warps);
    else if (sp.pair16) run<true>(db, sp, qc, pq, warps);
    else run<false>(db, sp, qc, pq, warps);

    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    const int32_t p16 = sp.pair16;
    fwrite(scores.data(), sizeof(int32_t), (size_t)n, o);
    fwrite(cells.data(), sizeof(int64_t), (size_t)n, o);
    fwrite(&p16, sizeof(p16), 1, o);
    fwrite(&long_end, sizeof(long_end), 1, o);
    fclose(o);
    return 0;
}
