// hs_scan.cu -- the database scan (every pair's score) and the alignment
// replay of the ranked hits: the database-search form of Fig. 1
// (Sec. III.B.3) for one query (plain) or many (batched), and the
// full-slide form (Fig. 1 as printed, several rounds).
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "hs_device.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// Profile preparation: both role profiles (reversed and forward query) into
// global memory, once per search; the scan CTAs copy theirs into shared
// memory and the replay reads them in place.  Batched: blockIdx.y = query.
// ---------------------------------------------------------------------------
struct ProfileJob {
    const uint8_t *queries;       // letters of all queries
    const int64_t *qoffsets;      // nullptr: one query of length qlen at queries
    const int64_t *prof_off;      // word offset of each query's profiles (batched)
    int32_t qlen;
    uint32_t *prof;
    int32_t *status;              // HS_EINVAL is recorded here for a letter code >= kNSym
    int32_t *init_scores;         // full-slide mode: [n_init] set to INT_MIN (nullptr: none)
    int64_t *init_cells;          // full-slide mode: [n_init] set to 0 (nullptr: none)
    int64_t n_init;
};

__global__ void profile_kernel(ProfileJob job, KParams kp)
{
    __shared__ int8_t msm[kNSym * kNSym];
    for (int i = threadIdx.x; i < kNSym * kNSym; i += blockDim.x) msm[i] = kp.m[i];
    __syncthreads();
    const uint8_t *q = job.queries;
    int qlen = job.qlen;
    uint32_t *prof = job.prof;
    if (job.qoffsets) {
        const int qi = blockIdx.y;
        q += job.qoffsets[qi];
        qlen = (int)(job.qoffsets[qi + 1] - job.qoffsets[qi]);
        prof += job.prof_off[qi];
    }
    // Device-resident queries reach the library unchecked: a code outside the
    // alphabet is reported through the status word and scores as a zero
    // column (profile_word_value) instead of indexing past the matrix.
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < qlen; i += gridDim.x * blockDim.x)
        if (q[i] >= kNSym && job.status) atomicCAS(job.status, (int32_t)HS_OK, (int32_t)HS_EINVAL);
    const int R = profile_stride(qlen);
    const int64_t words = profile_words(qlen);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * words;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const bool rev = idx < words;
        const int64_t i = rev ? idx : idx - words;
        const int a = (int)(i / R), s = (int)(i - (int64_t)a * R);
        prof[idx] = profile_word_value(q, qlen, rev, msm, kp.s.bias, a, s);
    }
    if (job.init_scores)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < job.n_init;
             i += (int64_t)gridDim.x * blockDim.x) {
            job.init_scores[i] = INT_MIN;
            if (job.init_cells) job.init_cells[i] = 0;
        }
}

// ---------------------------------------------------------------------------
// The pair loop shared by the plain and batched scans.  Every lane of a warp
// owns one pair: its O(1) state (Sec. III.B.4) -- positions, step, score,
// best round, size factors, one cached Philox block -- sits in that lane's
// registers, so the step bookkeeping of 32 pairs runs as one SIMT
// instruction stream.  Each round of the loop plans one step for every held
// pair.  With 16-bit pair sums the chunks of every step that joins the flat
// list are dealt to the warp's 32 lanes as units (see run_pairs); the other
// steps (few long chunks) are scanned one at a time by the whole warp on a
// lane grid (coop_scan_t), reading the step's plan from the warp's
// shared-memory plan slots.  With 32-bit sums (wide matrices) small steps
// (at most kLocalIters chunk iterations) are scored by their own lane and
// the rest on the lane grid.  Positions come from a queue over the
// length-ordered database (longest first); targets of >= kLongLen letters
// are taken one per warp (only lane 0 holds a pair) so each gets the warp
// alone.  The full-slide mode's loops (run_full_items, run_full_pairs)
// follow at the end of this part.
// ---------------------------------------------------------------------------
constexpr int kLocalIters = 64;
// flattened scan (16-bit pair sums): a step joins the unit list when it has
// at least sp.flat_min_chunks chunks or at most sp.flat_max_iters iterations
// per chunk; the rest (few long chunks) get the warp's lane grid

struct QueryCtx {
    const uint32_t *prof_rev;       // profile for pairs where the query is the small sequence
    const uint32_t *prof_fwd;       // ... and where it is the large one
    int32_t *scores;                // [n] by database index
    int64_t *cells;                 // optional [n]
};

struct Lane {                       // one pair held by one lane
    int32_t d;                      // database index (< 2^31 by hs_db_load), -1 = empty
    const uint8_t *t;
    int32_t nl, ns, qsmall;
    int32_t Lp, Sp, step, score, best, round;
    uint32_t lf, sf;
    int64_t cells;
    int32_t blk;                    // Philox block cached in w0..w3
    uint64_t w0, w1, w2, w3;
};

__device__ __forceinline__ uint32_t lane_draw(Lane &L, const SParams &sp, uint64_t i)
{
    const int32_t b = (int32_t)(i >> 4);
    if (b != L.blk) {
        uint64_t o[4];
        philox4x64_10((uint64_t)((int64_t)L.d + sp.index_base), (uint64_t)L.round, (uint64_t)b, 0, sp.seed, 0, o);
        L.w0 = o[0]; L.w1 = o[1]; L.w2 = o[2]; L.w3 = o[3];
        L.blk = b;
    }
    const unsigned wi = (unsigned)(i >> 2) & 3u;
    const uint64_t w = wi == 0 ? L.w0 : wi == 1 ? L.w1 : wi == 2 ? L.w2 : L.w3;
    return (uint32_t)(w >> (48 - 16 * (unsigned)(i & 3))) & 0xFFFFu;
}

// Start round L.round: lf = MAX(minFactor, LFactor*random()), sf likewise.
__device__ __forceinline__ void lane_start_round(Lane &L, const SParams &sp)
{
    L.blk = -1;
    uint32_t lf = (uint32_t)(((uint64_t)sp.lf_q16 * lane_draw(L, sp, 0)) >> 16);
    uint32_t sf = (uint32_t)(((uint64_t)sp.sf_q16 * lane_draw(L, sp, 1)) >> 16);
    L.lf = max(lf, sp.minf_q16);
    L.sf = max(sf, sp.minf_q16);
    L.Lp = 0; L.Sp = 0; L.step = 0; L.score = 0;
}

// Finish every round whose loop has ended (Fig. 1: the leftover letters go
// against gaps; AlignSequences keeps the first best round), then the pair.
__device__ __forceinline__ void lane_settle(Lane &L, const SParams &sp, const QueryCtx &qc)
{
    while (L.d >= 0 && !(L.Lp < L.nl && L.Sp < L.ns)) {
        L.score -= sp.pgp * ((L.nl - L.Lp) + (L.ns - L.Sp));
        if (L.score > L.best) L.best = L.score;
        L.round++;
        if (L.round < sp.rounds) {
            lane_start_round(L, sp);
        } else {
            qc.scores[L.d] = L.best;
            if (qc.cells) qc.cells[L.d] = L.cells;
            L.d = -1;
        }
    }
}

// A warp's step shared with the idle warps of its CTA (the end of a scan,
// when one long pair is left on a warp while the others have run out of
// pairs).  claim = units of the step << 32 | the next unit to hand out;
// whoever takes a pass of 32 units (the owner or a helper) scores it, folds
// its best key into `key` and then adds its units to `done`.  The owner
// publishes a step only after the previous one is done, and a helper reads
// the descriptor only after a claim below the step's units, so the
// descriptor it reads is that step's.
struct HelpBoard {
    unsigned long long claim;
    uint4 desc;
    uint32_t key, done;
};

// Per-warp shared slots of the flattened scan, in rank order: each flat
// step's descriptor and best key, and each lane's rank.
struct FlatSlots {
    uint4 desc[32];
    uint32_t key[32];
    int32_t rank[32];
};

// Sharing between the warps of one CTA: every warp's slots and board (warp
// w's at slots + w, boards + w), the warps still working on pairs of their
// own, and the status word a wait that runs out records HS_ETIMEOUT in.
struct Help {
    FlatSlots *slots;
    HelpBoard *boards;
    int nw;
    unsigned *live;
    int32_t *status;
};
constexpr uint64_t kHelpWaitNs = 2000000000ull;     // 2 s: a helper's wait for work; an owner's for its helpers

__device__ __forceinline__ uint64_t help_now_ns()
{
#if defined(__CUDA_ARCH__)
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
#elif defined(HS_HOST_EMULATION)
    return emu_now_ns();
#else
    return 0;                       // the device compiler's host pass: never called
#endif
}

template <class T> __device__ __forceinline__ T help_load(const T *p)
{
#if defined(HS_HOST_EMULATION)
    return __atomic_load_n(p, __ATOMIC_ACQUIRE);
#else
    return *reinterpret_cast<const volatile T *>(p);
#endif
}

// One pass of a shared step: units base .. base + 31 of tot, by the calling
// warp; the pass's best key goes into the board before its units count as done.
__device__ __forceinline__ void help_pass(HelpBoard &bd, const uint4 &d, unsigned base, unsigned tot,
                                          const QueryCtx &qc, int R, const SParams &sp, int lane)
{
    const unsigned u = base + (unsigned)lane;
    const uint32_t key = u < tot ? desc_key(qc.prof_rev, qc.prof_fwd, R, d, 4 * (int)u, sp.flush) : 0u;
    const uint32_t m = __reduce_max_sync(0xFFFFFFFFu, key);
    if (lane == 0) {
        atomicMax(&bd.key, m);
        __threadfence_block();
        atomicAdd(&bd.done, min(32u, tot - base));
    }
}

__device__ __forceinline__ void help_fail(const Help *hp)
{
    if (hp->status) atomicCAS(hp->status, (int32_t)HS_OK, (int32_t)HS_ETIMEOUT);
}

// The owner's side: publish the lone flat step (slot 0), take passes like
// any helper, wait for the passes others took, leave the best key in slot 0.
__device__ __forceinline__ void share_step(const Help *hp, FlatSlots *fs, unsigned tot, const QueryCtx &qc, int R,
                                           const SParams &sp, int lane)
{
    HelpBoard &bd = hp->boards[fs - hp->slots];
    const uint4 d = fs->desc[0];
    if (lane == 0) {
        bd.desc = d;
        bd.key = 0u;
        bd.done = 0u;
        __threadfence_block();
        atomicExch(&bd.claim, (unsigned long long)tot << 32);
    }
    __syncwarp();
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&bd.claim, 32ull);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        if ((unsigned)c >= tot) break;
        help_pass(bd, d, (unsigned)c, tot, qc, R, sp, lane);
    }
    if (lane == 0) {
        const uint64_t t0 = help_now_ns();
        while (help_load(&bd.done) < tot) {
            if (help_now_ns() - t0 > kHelpWaitNs) { help_fail(hp); break; }
        }
        __threadfence_block();
        fs->key[0] = help_load(&bd.key);
    }
    __syncwarp();
}

// A warp out of pairs: take passes of the other warps' shared steps until
// every warp of the CTA is out of pairs (after which none is published), or
// until it has found none for kHelpWaitNs.
__device__ __forceinline__ void help_out(const Help *hp, const QueryCtx &qc, int R, const SParams &sp, int lane)
{
    __syncwarp();
    if (lane == 0) atomicAdd(hp->live, 0xFFFFFFFFu);
    uint64_t t0 = help_now_ns();
    unsigned nap = 256;                 // ns between looks, doubled up to 4 us while there is no work
    for (;;) {
        unsigned long long c = 0;
        if (lane < hp->nw) c = help_load(&hp->boards[lane].claim);
        const unsigned open_boards = __ballot_sync(0xFFFFFFFFu, lane < hp->nw && (unsigned)c < (unsigned)(c >> 32));
        if (open_boards) {
            HelpBoard &bd = hp->boards[__ffs((int)open_boards) - 1];
            unsigned long long x = 0;
            if (lane == 0) x = atomicAdd(&bd.claim, 32ull);
            x = __shfl_sync(0xFFFFFFFFu, x, 0);
            __syncwarp();
            const unsigned base = (unsigned)x, tot = (unsigned)(x >> 32);
            if (base < tot) help_pass(bd, bd.desc, base, tot, qc, R, sp, lane);
            t0 = help_now_ns();
            nap = 256;
            continue;
        }
        unsigned live = 0;
        if (lane == 0) live = help_load(hp->live);
        live = __shfl_sync(0xFFFFFFFFu, live, 0);
        if (live == 0) break;
        // helping is optional (an owner takes every pass nobody else
        // takes), so a helper that has found no work for a while leaves
        bool late = false;
        if (lane == 0) late = help_now_ns() - t0 > kHelpWaitNs;
        if (__shfl_sync(0xFFFFFFFFu, late, 0)) break;
        __nanosleep(nap);
        nap = min(2 * nap, 4096u);
    }
}

// Fold a pass's unit keys into their steps' keys.  Units of one step sit in
// adjacent lanes; lanes past the list hold key 0, which no maximum notices.
// A pass where no step begins after lane 0 (starts: the pass's start mask)
// has one owner: it takes one warp maximum and one atomic, the others one
// atomic per unit.
__device__ __forceinline__ void fold_keys(FlatSlots *fs, unsigned starts, int owner, bool valid, uint32_t key,
                                          int lane)
{
    if ((starts >> 1) == 0u) {
        const uint32_t m = __reduce_max_sync(0xFFFFFFFFu, key);
        if (lane == 0) atomicMax(&fs->key[owner], m);
    } else if (valid) {
        atomicMax(&fs->key[owner], key);
    }
}

// Queue positions [begin, end) of the length order; [begin, long_end) long.
struct PosQueue {
    int64_t begin, long_end, end;
    unsigned *ctr;                  // global or shared counter of handed-out positions
    unsigned lanes;                 // lanes a warp fills with pairs (bit mask; a small database spreads thin)
};

// kHelp: the warps of the CTA share large lone steps at the scan's end (hp
// set).  It is a separate build of the loop because the sharing code, even
// unused, costs the 80-register loop about 2% (measured), so the library
// takes it only for databases with many very long targets, where one pair's
// chain of steps can outlast the rest of the scan.
template <bool P16, bool kHelp = false>
__device__ __forceinline__ void run_pairs(const DbView &db, const SParams &sp, const QueryCtx &qc,
                                          const PosQueue &qu, Plan *plans, FlatSlots *fs, int lane,
                                          const Help *hp = nullptr)
{
    const int R = profile_stride(sp.qlen);
    const unsigned lt_mask = (1u << lane) - 1u;
    Lane L = {};
    L.d = -1;
    L.t = db.codes;
    L.best = INT_MIN;
    int phase = qu.long_end > qu.begin ? 0 : 1;       // 0: one long target per warp
    bool open = qu.end > qu.begin;
    for (;;) {
        // refill empty lanes from the queue
        if (open) {
            unsigned need = __ballot_sync(0xFFFFFFFFu, L.d < 0) & qu.lanes;
            if (phase == 0) need &= 1u;
            if (need) {
                const int m = __popc(need);
                long long base = 0;
                if (lane == 0) base = (long long)qu.begin + (long long)atomicAdd(qu.ctr, (unsigned)m);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (base + m >= qu.end) open = false;
                if (phase == 0 && base >= qu.long_end) phase = 1;
                const long long pos = base + __popc(need & lt_mask);
                if (((need >> lane) & 1u) && pos < qu.end) {
                    L.d = db.order[pos];
                    const int64_t off = db.offsets[L.d];
                    const int32_t tlen = (int32_t)(db.offsets[L.d + 1] - off);
                    L.t = db.codes + off;
                    L.qsmall = tlen >= sp.qlen;            // the target is large on ties
                    L.nl = L.qsmall ? tlen : sp.qlen;
                    L.ns = L.qsmall ? sp.qlen : tlen;
                    L.round = 0;
                    L.best = INT_MIN;
                    L.cells = 0;
                    lane_start_round(L, sp);
                    lane_settle(L, sp, qc);                 // empty small sequence
                }
            }
        }
        __syncwarp();
        const bool busy = L.d >= 0;
        if (!open && __ballot_sync(0xFFFFFFFFu, busy) == 0) {
            if constexpr (P16 && kHelp) help_out(hp, qc, R, sp, lane);      // only flat steps are shared
            break;
        }

        // plan one step per held pair (Fig. 1's Align: ls and ss, A6)
        Plan g = {L.t, L.Lp, L.Sp, 1, 1, L.qsmall, 0, 0, 0};
        int32_t vmax = 0, kstar = 0;
        bool local = false;                 // scanned by its own lane (wide matrices)
        bool flat = false;                  // scanned as units of the flattened list
        if (busy) {
            const int32_t Lrem = L.nl - L.Lp, Srem = L.ns - L.Sp;
            const int32_t ls = max((int32_t)(((uint64_t)Lrem * L.lf) >> 16), 1);
            const uint64_t u = lane_draw(L, sp, 2 + (uint64_t)L.step);
            const int64_t ssw = (int64_t)(((uint64_t)Srem * L.sf * u) >> 32);
            g.ls = ls;
            g.ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)min(Srem, ls)));
            const int32_t nchunk = (ls - g.ss + 4) >> 2;
            const int32_t niter = g.ss + (L.qsmall ? 3 : 0);
            if constexpr (P16) {
                flat = ls - g.ss < 65536 && (nchunk >= sp.flat_min_chunks || niter <= sp.flat_max_iters);
                if (!flat) plan_grid(g);
            } else {
                local = (int64_t)nchunk * niter <= kLocalIters;
                if (local) lane_scan_t<P16>(L.qsmall ? qc.prof_rev : qc.prof_fwd, R, sp.qlen, g, sp.bias, sp.flush,
                                            vmax, kstar);
                else plan_grid(g);
            }
        }
        if constexpr (P16) {
            // Flattened scan: the chunks of every flat step form one list of
            // units dealt to the 32 lanes, 32 at a time.  Steps are ranked by
            // role, then by iterations per unit, most first (a bitonic sort
            // across the warp), so that the units sharing a pass have similar
            // trip counts and the last pass, the one only partly filled,
            // holds the shortest units; flat slot r holds the descriptor and
            // key of the step of rank r.  A
            // unit's lane finds its step from the pass's start mask (below)
            // and scores its chunk; the pass folds the chunk keys into
            // the steps' keys.
            const int units = flat ? (g.ls - g.ss + 4) >> 2 : 0;
            const uint32_t iters = (uint32_t)min(g.ss + 3 * g.qsmall, (1 << 24) - 1);
            uint32_t sk = flat ? ((uint32_t)g.qsmall << 30) | ((0xFFFFFFu - iters) << 5) | (uint32_t)lane
                               : 0x80000000u | (uint32_t)lane;
            for (int k = 2; k <= 32; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, sk, j);
                    const bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
                    sk = take_min ? min(sk, o) : max(sk, o);
                }
            }
            const int src = (int)(sk & 31u);        // the lane whose step has rank `lane`
            const int ru = __shfl_sync(0xFFFFFFFFu, units, src);
            int incl = ru;
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += x;
            }
            const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            fs->rank[src] = lane;
            fs->key[lane] = 0u;
            __syncwarp();
            const int slot = fs->rank[lane];
            if (flat) fs->desc[slot] = flat_desc(g, sp.qlen);
            else if (busy) plans[lane] = g;
            __syncwarp();
            // Owners without a search: this lane, as rank `lane`, begins its
            // step's units at incl - ru; one OR over the warp marks the lanes
            // of a pass where a step begins, and a unit's owner is the last
            // owner of the previous pass plus the beginnings up to its lane.
            const int my_u0 = incl - ru;
            int carry = -1, carry_u0 = 0;           // the last unit's owner and its first unit
            // a lone large step is shared once some warp of the CTA is out of
            // pairs (only at the scan's end; until then the owner takes every
            // pass through the plain loop below)
            bool share = false;
            if constexpr (kHelp) {
                if (total >= sp.help_min_units && __popc(__ballot_sync(0xFFFFFFFFu, flat)) == 1) {
                    unsigned live = 0;
                    if (lane == 0) live = help_load(hp->live);
                    share = __shfl_sync(0xFFFFFFFFu, live, 0) < (unsigned)hp->nw;
                }
                if (share) share_step(hp, fs, (unsigned)total, qc, R, sp, lane);
            }
            for (int base = 0; base < (share ? 0 : total); base += 32) {
                const int u = base + lane;
                const bool valid = u < total;
                uint32_t key = 0u;
                const unsigned starts = __reduce_or_sync(0xFFFFFFFFu, start_bit(my_u0, ru, base));
                const int owner = pass_owner(carry, starts, lane);
                const int first = pass_first_unit(carry_u0, starts, base, lane);
                carry_u0 = pass_first_unit(carry_u0, starts, base, 31);     // lane 31's, for the next pass
                carry = pass_owner(carry, starts, 31);
                if (valid) {
                    const uint4 d = fs->desc[owner];
                    key = desc_key(qc.prof_rev, qc.prof_fwd, R, d, 4 * (u - first), sp.flush);
                }
                fold_keys(fs, starts, owner, valid, key, lane);
            }
            __syncwarp();
            if (flat) {
                const uint32_t key = fs->key[slot];
                vmax = (int32_t)(key >> 16) - sp.bias * g.ss;
                kstar = (int32_t)(0xFFFFu - (key & 0xFFFFu));
            }
        } else {
            if (busy && !local) plans[lane] = g;
        }
        __syncwarp();
        // the other steps, one pair at a time, by the whole warp
        unsigned coop = __ballot_sync(0xFFFFFFFFu, busy && !local && !flat);
        while (coop) {
            const int i = __ffs(coop) - 1;
            coop &= coop - 1;
            const Plan h = plans[i];
            int32_t v, k;
            coop_scan_t<P16>(h.qsmall ? qc.prof_rev : qc.prof_fwd, R, sp.qlen, h, sp.bias, sp.flush, lane, v, k);
            if (lane == i) { vmax = v; kstar = k; }
        }
        // consume (Fig. 1: drop what the step took from both) and score incrementally (A17)
        if (busy) {
            const int64_t nshift = g.ls - g.ss + 1;
            L.cells += nshift * g.ss + (sp.pack_shifts ? nshift << 40 : 0);
            int32_t gap = 0;
            if (kstar > 0) gap = (L.step == 0) ? sp.pgp * kstar : sp.gop + (kstar - 1) * sp.gep;
            L.score += vmax - gap;
            L.Lp += kstar + g.ss;
            L.Sp += g.ss;
            L.step++;
            lane_settle(L, sp, qc);
        }
        __syncwarp();
    }
}

// Full-slide mode (pair-wise form).  A pair's rounds are independent runs of
// Align (AlignSequences, Fig. 1) whose draws are keyed by (index, round), so
// a work item is one (position, round): a long pair's rounds run on many
// warps at once instead of one after another.  Items go out position-major
// over the length order (the longest pairs' rounds first); each folds its
// round's score into the pair's by atomicMax (the best of the rounds; the
// winning round is found again by the replay) and its cells into the
// pair's count by atomicAdd, so scores must start at INT_MIN and counts at
// 0 (profile_kernel clears them).
struct FullQueue {
    int64_t begin, end;             // positions [begin, end) of the length order
    unsigned long long *ctr;        // items handed out
    const uint32_t *prof_rev, *prof_fwd;
    int64_t long_end;               // run_full_pairs: positions [begin, long_end) are taken one item per warp
};

__device__ __forceinline__ void run_full_items(const DbView &db, const SParams &sp, const FullQueue &qu,
                                               int32_t *scores, int64_t *cells_out, int lane)
{
    const unsigned long long rounds = (unsigned)sp.rounds;
    const unsigned long long items = (unsigned long long)(qu.end - qu.begin) * rounds;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(qu.ctr, 1ull);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= items) break;
        const unsigned long long pi = it / rounds;
        const int r = (int)(it - pi * rounds);
        const int64_t d = db.order[qu.begin + (int64_t)pi];
        const int64_t off = db.offsets[d];
        PairCtx c;
        c.t = db.codes + off;
        c.tlen = (int32_t)(db.offsets[d + 1] - off);
        c.qlen = sp.qlen;
        c.qsmall = c.tlen >= sp.qlen;
        c.prof = c.qsmall ? qu.prof_rev : qu.prof_fwd;
        c.S = profile_stride(sp.qlen);
        int64_t cells = 0;
        const int32_t s = align_round_full<false>(c, sp, (uint64_t)d, r, lane, cells, nullptr, nullptr);
        if (lane == 0) {
            atomicMax(&scores[d], s);
            if (cells_out) atomicAdd(reinterpret_cast<unsigned long long *>(&cells_out[d]), (unsigned long long)cells);
        }
    }
}

// Full-slide mode with lane-owned items (16-bit pair sums, a matrix with a
// non-negative entry): every lane of a warp holds one (position, round)
// item -- a long pair's rounds sit in neighbouring lanes -- in the database
// form's lane state plus the round's RunScore (F4).  Each loop round plans
// one full-slide step per item (F2: ss up to Srem, not ls), deals the chunks
// of all flat steps over the warp as in run_pairs (ranked by role and trip
// count, owners from the pass start masks, keys folded by warp maximum or
// shared atomics: full_desc_key), scans the others warp-wide
// (full_scan_t), and consumes every step by F3.  A finished round folds
// its score and cells into the pair's by atomics, as run_full_items does.
__device__ __forceinline__ void run_full_pairs(const DbView &db, const SParams &sp, const QueryCtx &qc,
                                               const FullQueue &fq, unsigned lanes, FlatSlots *fs, Plan *plans,
                                               int lane)
{
    const int R = profile_stride(sp.qlen);
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long rounds = (unsigned)sp.rounds;
    const unsigned long long items = (unsigned long long)(fq.end - fq.begin) * rounds;
    const unsigned long long long_items = (unsigned long long)(max(fq.long_end, fq.begin) - fq.begin) * rounds;
    Lane L = {};
    L.d = -1;
    L.t = db.codes;
    RunScore rs;
    rs.init();
    bool open = items > 0;
    bool alone = long_items > 0;            // a long target's rounds: one per warp, so each has the warp alone
    for (;;) {
        if (open) {
            unsigned need = __ballot_sync(0xFFFFFFFFu, L.d < 0) & lanes;
            if (alone) need &= 1u;
            if (need) {
                const int m = __popc(need);
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(fq.ctr, (unsigned long long)m);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (base + m >= items) open = false;
                if (base >= long_items) alone = false;
                const unsigned long long it = base + (unsigned long long)__popc(need & lt_mask);
                if (((need >> lane) & 1u) && it < items) {
                    const unsigned long long pi = it / rounds;
                    L.d = db.order[fq.begin + (int64_t)pi];
                    L.round = (int32_t)(it - pi * rounds);
                    const int64_t off = db.offsets[L.d];
                    const int32_t tlen = (int32_t)(db.offsets[L.d + 1] - off);
                    L.t = db.codes + off;
                    L.qsmall = tlen >= sp.qlen;
                    L.nl = L.qsmall ? tlen : sp.qlen;
                    L.ns = L.qsmall ? sp.qlen : tlen;
                    L.cells = 0;
                    lane_start_round(L, sp);
                    rs.init();
                }
            }
        }
        // a round whose loop has ended (or never began: an empty sequence)
        // settles: the rest of each sequence against gaps, then the fold
        if (L.d >= 0 && !(L.Lp < L.nl && L.Sp < L.ns)) {
            rs.gap(1, L.nl - L.Lp);
            rs.gap(0, L.ns - L.Sp);
            rs.finish(sp);
            atomicMax(&qc.scores[L.d], rs.score);
            if (qc.cells) atomicAdd(reinterpret_cast<unsigned long long *>(&qc.cells[L.d]), (unsigned long long)L.cells);
            L.d = -1;
        }
        __syncwarp();
        const bool busy = L.d >= 0;
        if (__ballot_sync(0xFFFFFFFFu, busy) == 0) {
            if (!open) break;
            continue;                       // every held round settled: refill
        }

        Plan g = {L.t, L.Lp, L.Sp, 1, 1, L.qsmall, 0, 0, 0};
        bool flat = false;
        if (busy) {
            const int32_t Lrem = L.nl - L.Lp, Srem = L.ns - L.Sp;
            g.ls = max((int32_t)(((uint64_t)Lrem * L.lf) >> 16), 1);
            const uint64_t u = lane_draw(L, sp, 2 + (uint64_t)L.step);
            const int64_t ssw = (int64_t)(((uint64_t)Srem * L.sf * u) >> 32);
            g.ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)Srem));                      // F2
            const int32_t nchunk = (g.ls + g.ss - 1 + 3) >> 2;
            const int32_t niter = g.ss + (L.qsmall ? 3 : 0);
            flat = g.ls + g.ss - 1 <= 65535 && (nchunk >= sp.flat_min_chunks || niter <= sp.flat_max_iters);
        }
        int32_t vmax = 0, kstar = 0;
        {
            const int units = flat ? (g.ls + g.ss - 1 + 3) >> 2 : 0;
            const uint32_t iters = (uint32_t)min(g.ss + 3 * g.qsmall, (1 << 24) - 1);
            uint32_t sk = flat ? ((uint32_t)g.qsmall << 30) | ((0xFFFFFFu - iters) << 5) | (uint32_t)lane
                               : 0x80000000u | (uint32_t)lane;
            for (int k = 2; k <= 32; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, sk, j);
                    const bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
                    sk = take_min ? min(sk, o) : max(sk, o);
                }
            }
            const int src = (int)(sk & 31u);
            const int ru = __shfl_sync(0xFFFFFFFFu, units, src);
            int incl = ru;
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += x;
            }
            const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            fs->rank[src] = lane;
            fs->key[lane] = 0u;
            __syncwarp();
            const int slot = fs->rank[lane];
            if (flat) fs->desc[slot] = full_desc(g, sp.qlen);
            else if (busy) plans[lane] = g;
            __syncwarp();
            const int my_u0 = incl - ru;
            int carry = -1, carry_u0 = 0;
            for (int base = 0; base < total; base += 32) {
                const int u = base + lane;
                const bool valid = u < total;
                uint32_t key = 0u;
                const unsigned starts = __reduce_or_sync(0xFFFFFFFFu, start_bit(my_u0, ru, base));
                const int owner = pass_owner(carry, starts, lane);
                const int first = pass_first_unit(carry_u0, starts, base, lane);
                carry_u0 = pass_first_unit(carry_u0, starts, base, 31);
                carry = pass_owner(carry, starts, 31);
                if (valid) {
                    const uint4 d = fs->desc[owner];
                    const int ss = (int)(d.z >> 16);
                    key = full_desc_key(qc.prof_rev, qc.prof_fwd, R, sp.qlen, d, 4 * (u - first) - (ss - 1),
                                        sp.bias, sp.flush);
                }
                fold_keys(fs, starts, owner, valid, key, lane);
            }
            __syncwarp();
            if (flat) {
                const uint32_t key = fs->key[slot];
                vmax = (int32_t)(key >> 16) - sp.bias * g.ss;
                kstar = (int32_t)(0xFFFFu - (key & 0xFFFFu)) - (g.ss - 1);
            }
        }
        // the other steps, one item at a time, by the whole warp
        unsigned coop = __ballot_sync(0xFFFFFFFFu, busy && !flat);
        while (coop) {
            const int i = __ffs(coop) - 1;
            coop &= coop - 1;
            const Plan h = plans[i];
            int32_t v, k;
            full_scan_t<true>(h.qsmall ? qc.prof_rev : qc.prof_fwd, R, sp.qlen, h, sp.bias, sp.flush, lane, v, k);
            if (lane == i) { vmax = v; kstar = k; }
        }
        // consume (F3: leading overhang, overlap, trailing overhang of small)
        if (busy) {
            L.cells += (int64_t)g.ls * g.ss;
            const int32_t j0 = max(0, -kstar), j1 = min(g.ss, g.ls - kstar);
            rs.gap(0, j0);
            rs.gap(1, max(kstar, 0));
            rs.match(vmax, sp);
            rs.gap(0, g.ss - j1);
            L.Lp += kstar + j1;
            L.Sp += g.ss;
            L.step++;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Plain scan: a persistent grid over one queue of the whole database.
// ---------------------------------------------------------------------------
struct ScanQueue {
    int64_t begin, long_end, end;
    unsigned *ctr;
    int32_t *status;                // HS_ETIMEOUT if a wait between warps runs out
    unsigned long long *items;      // full-slide mode: (position, round) items handed out
    int64_t smem_words;             // profile words staged into shared memory
    int rev_off, fwd_off;           // word offsets of the two role profiles
    unsigned lanes;                 // PosQueue::lanes
};

// The lanes a warp fills: all 32 when the queue holds at least 32 pairs per
// resident warp; fewer for a small database, so that its pairs spread over
// all the warps (a warp's steps still deal their units to all 32 lanes)
// instead of crowding a few.
static unsigned lanes_for(int64_t pairs, int64_t warps)
{
    const int64_t per = warps > 0 ? (pairs + warps - 1) / warps : 32;
    return per >= 32 ? 0xFFFFFFFFu : (1u << (unsigned)(per < 1 ? 1 : per)) - 1u;
}

// The 8-warp scan CTA (static slots, 3 CTAs per SM), used for the
// database-order schedule; the length-order launches use scan_wide_kernel.
constexpr int kScanWarps = 8;

// kSmem: the profiles are staged in shared memory (known to the compiler, so
// every profile read is a shared load); otherwise they are read in place from
// global memory (database-order schedule with a query too long for both
// roles to fit).  P16: 16-bit chunk sums (SParams::pair16).
template <bool kSmem, bool P16>
__global__ void __launch_bounds__(kScanWarps * 32, 3)
scan_kernel(DbView db, ScanQueue qu, const uint32_t *__restrict__ prof_g, SParams sp,
            int32_t *__restrict__ scores, int64_t *__restrict__ cells_out)
{
    extern __shared__ uint4 smem_raw[];
    __shared__ Plan plans[kScanWarps][32];
    __shared__ FlatSlots flat_slots[kScanWarps];
    const uint32_t *prof = prof_g;
    if (kSmem) {
        const int64_t n16 = qu.smem_words / 4;          // profile words are a multiple of 4
        const uint4 *src = reinterpret_cast<const uint4 *>(prof_g);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) smem_raw[i] = src[i];
        __syncthreads();
        prof = reinterpret_cast<const uint32_t *>(smem_raw);
    }
    QueryCtx qc;
    qc.prof_rev = prof + qu.rev_off;
    qc.prof_fwd = prof + qu.fwd_off;
    qc.scores = scores;
    qc.cells = cells_out;
    const PosQueue pq = {qu.begin, qu.long_end, qu.end, qu.ctr, qu.lanes};
    run_pairs<P16>(db, sp, qc, pq, plans[threadIdx.x >> 5], &flat_slots[threadIdx.x >> 5], threadIdx.x & 31);
}

// The same scan for one role's profile of a long query (one role per launch):
// one CTA per SM with kWarps warps, the plan and flat-step slots in dynamic
// shared memory after the profile, so that the SM keeps as many warps as the
// fused short-query launch although the profile takes most of its memory.
template <bool P16, int kWarps, bool kHelp>
__global__ void __launch_bounds__(kWarps * 32, 1)
scan_wide_kernel(DbView db, ScanQueue qu, const uint32_t *__restrict__ prof_g, SParams sp,
                 int32_t *__restrict__ scores, int64_t *__restrict__ cells_out)
{
    extern __shared__ uint4 smem_raw[];
    const int64_t n16 = qu.smem_words / 4;
    const uint4 *src = reinterpret_cast<const uint4 *>(prof_g);
    Plan *plans = reinterpret_cast<Plan *>(smem_raw + n16);
    FlatSlots *slots = reinterpret_cast<FlatSlots *>(plans + kWarps * 32);
    HelpBoard *boards = reinterpret_cast<HelpBoard *>(slots + kWarps);
    unsigned *live = reinterpret_cast<unsigned *>(boards + kWarps);
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) smem_raw[i] = src[i];
    if (kHelp) {
        if (threadIdx.x < kWarps) {
            boards[threadIdx.x].claim = 0ull;           // no step to share
            boards[threadIdx.x].done = 0u;
        }
        if (threadIdx.x == 0) *live = kWarps;
    }
    __syncthreads();
    const uint32_t *prof = reinterpret_cast<const uint32_t *>(smem_raw);
    const Help help = {slots, boards, kWarps, live, qu.status};
    QueryCtx qc;
    qc.prof_rev = prof + qu.rev_off;
    qc.prof_fwd = prof + qu.fwd_off;
    qc.scores = scores;
    qc.cells = cells_out;
    const PosQueue pq = {qu.begin, qu.long_end, qu.end, qu.ctr, qu.lanes};
    const int w = threadIdx.x >> 5;
    run_pairs<P16, kHelp>(db, sp, qc, pq, plans + 32 * w, slots + w, threadIdx.x & 31, &help);
}

constexpr size_t kWarpSlotBytes = 32 * sizeof(Plan) + sizeof(FlatSlots);
constexpr size_t kCtaSlotBytes = 16;                 // the wide kernel's live-warp count
constexpr size_t kHelpSlotBytes = sizeof(HelpBoard);  // and its warps' boards

typedef void (*ScanKernelFn)(DbView, ScanQueue, const uint32_t *, SParams, int32_t *, int64_t *);

// Launch configuration queries, cached per device and (kernel, threads,
// shared memory): the opt-in shared-memory limit, the dynamic shared-memory
// attribute last set and the resident CTAs per SM.  A search makes the same
// few launches every time, so after the first one it queries nothing.
static std::mutex g_launch_mu;

static int smem_optin()
{
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    cache[dev] = optin;
    return optin;
}

// Sets the kernel's dynamic shared-memory limit (when it grows) and returns
// its resident CTAs per SM for `threads` threads and `smem` bytes.
static cudaError_t launch_fit(const void *fn, int threads, size_t smem, int *per_sm)
{
    static std::map<std::tuple<int, const void *>, size_t> smem_set;
    static std::map<std::tuple<int, const void *, int, size_t>, int> occ;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    const auto ks = std::make_tuple(dev, fn);
    auto si = smem_set.find(ks);
    if (si == smem_set.end() || si->second < smem) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set[ks] = smem;
    }
    const auto ko = std::make_tuple(dev, fn, threads, smem);
    auto oi = occ.find(ko);
    if (oi != occ.end()) { *per_sm = oi->second; return cudaSuccess; }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
    if (e != cudaSuccess) return e;
    occ[ko] = *per_sm;
    return cudaSuccess;
}

// The widest CTA whose profile and per-warp slots fit one SM's shared memory
// (0: none; the 8-warp kernel with static slots is used).
static int wide_warps(int64_t smem_words)
{
    const int optin = smem_optin();
    if (optin <= 0) return 0;
    const size_t prof = (size_t)smem_words * 4;
    for (int w : {24, 12})
        if (prof + w * (kWarpSlotBytes + kHelpSlotBytes) + kCtaSlotBytes <= (size_t)optin) return w;
    return 0;
}

// help: the build whose warps share large lone steps (16-bit sums only)
static ScanKernelFn pick_wide_kernel(int warps, bool p16, bool help)
{
    if (warps == 24) return p16 ? (help ? scan_wide_kernel<true, 24, true> : scan_wide_kernel<true, 24, false>)
                                : scan_wide_kernel<false, 24, false>;
    return p16 ? (help ? scan_wide_kernel<true, 12, true> : scan_wide_kernel<true, 12, false>)
               : scan_wide_kernel<false, 12, false>;
}

static ScanKernelFn pick_scan_kernel(bool smem, bool p16)
{
    if (smem) return p16 ? scan_kernel<true, true> : scan_kernel<true, false>;
    return p16 ? scan_kernel<false, true> : scan_kernel<false, false>;
}

// Full-slide mode (pair-wise form): each warp takes (position, round) items
// (run_full_items) from the queue's 64-bit counter.  Three CTAs per SM (80
// registers, no spills): the steps' chains of dependent loads want warps.
template <bool kSmem>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 3)
scan_full_kernel(DbView db, ScanQueue qu, const uint32_t *__restrict__ prof_g, SParams sp,
                 int32_t *__restrict__ scores, int64_t *__restrict__ cells_out)
{
    extern __shared__ uint4 smem_raw[];
    const uint32_t *prof = prof_g;
    if (kSmem) {
        const int64_t n16 = qu.smem_words / 4;
        const uint4 *src = reinterpret_cast<const uint4 *>(prof_g);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) smem_raw[i] = src[i];
        __syncthreads();
        prof = reinterpret_cast<const uint32_t *>(smem_raw);
    }
    const FullQueue fq = {qu.begin, qu.end, qu.items, prof + qu.rev_off, prof + qu.fwd_off, qu.begin};
    run_full_items(db, sp, fq, scores, cells_out, threadIdx.x & 31);
}

// Full-slide mode, lane-owned items (run_full_pairs).
template <bool kSmem>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 2)
scan_full_lanes_kernel(DbView db, ScanQueue qu, const uint32_t *__restrict__ prof_g, SParams sp,
                       int32_t *__restrict__ scores, int64_t *__restrict__ cells_out)
{
    extern __shared__ uint4 smem_raw[];
    __shared__ Plan plans[kWarpsPerCta][32];
    __shared__ FlatSlots flat_slots[kWarpsPerCta];
    const uint32_t *prof = prof_g;
    if (kSmem) {
        const int64_t n16 = qu.smem_words / 4;
        const uint4 *src = reinterpret_cast<const uint4 *>(prof_g);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) smem_raw[i] = src[i];
        __syncthreads();
        prof = reinterpret_cast<const uint32_t *>(smem_raw);
    }
    QueryCtx qc;
    qc.prof_rev = prof + qu.rev_off;
    qc.prof_fwd = prof + qu.fwd_off;
    qc.scores = scores;
    qc.cells = cells_out;
    const FullQueue fq = {qu.begin, qu.end, qu.items, qc.prof_rev, qc.prof_fwd, qu.long_end};
    const int w = threadIdx.x >> 5;
    run_full_pairs(db, sp, qc, fq, qu.lanes, &flat_slots[w], plans[w], threadIdx.x & 31);
}

size_t scan_smem_bytes(int32_t qlen) { return (size_t)profile_words(qlen) * 4; }

// Several-CTA-per-SM kernels (database order, full-slide mode): both
// profiles share one launch when they fit twice per SM with room to spare.
static bool fuse_roles(int32_t qlen) { return 2 * scan_smem_bytes(qlen) <= 100 * 1024; }

cudaError_t launch_scan(const DbView &db, int64_t split, int64_t long_end, const uint8_t *d_query,
                        const KParams &kp, const Workspace &ws, int64_t *d_cells, int32_t *d_status, int num_sms,
                        cudaStream_t st, const ScanTrace *trace, int *launches, bool input_order,
                        bool share_steps)
{
    const int64_t words = profile_words(kp.s.qlen);
    ProfileJob job = {d_query, nullptr, nullptr, kp.s.qlen, ws.prof, d_status};
    if (kp.s.mode == HS_MODE_FULL) {
        job.init_scores = ws.scores;
        job.init_cells = d_cells;
        job.n_init = db.n;
    }
    profile_kernel<<<64, 256, 0, st>>>(job, kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int nl = 1;

    ScanQueue qs[2];
    const uint32_t *srcs[2];
    int nq = 0;
    if (input_order) {
        // one queue in database order, roles mixed, no long-target phase
        ScanQueue &q = qs[nq];
        q.begin = 0; q.end = db.n; q.long_end = 0;
        q.ctr = ws.counters + kQsLong;
        q.smem_words = fuse_roles(kp.s.qlen) ? 2 * words : 0;
        q.rev_off = 0; q.fwd_off = (int)words;
        srcs[nq++] = ws.prof;
    } else if (kp.s.mode == HS_MODE_FULL ? fuse_roles(kp.s.qlen) : wide_warps(2 * words) == 24) {
        // database form: both role profiles in one launch whenever they fit
        // beside 24 warps' slots (queries up to ~940 letters); the
        // full-slide kernels run several CTAs per SM and keep the 100 KB rule
        ScanQueue &q = qs[nq];
        q.begin = 0; q.end = db.n; q.long_end = min(long_end, split);
        q.ctr = ws.counters + kQsLong;
        q.smem_words = 2 * words; q.rev_off = 0; q.fwd_off = (int)words;
        srcs[nq++] = ws.prof;
    } else {
        if (split > 0) {
            ScanQueue &q = qs[nq];
            q.begin = 0; q.end = split; q.long_end = min(long_end, split);
            q.ctr = ws.counters + kQsLong;
            q.smem_words = words; q.rev_off = 0; q.fwd_off = 0;
            srcs[nq++] = ws.prof;
        }
        if (split < db.n) {
            ScanQueue &q = qs[nq];
            q.begin = split; q.end = db.n; q.long_end = split;   // every target is shorter than the query
            q.ctr = ws.counters + kQlLong;
            q.smem_words = words; q.rev_off = 0; q.fwd_off = 0;
            srcs[nq++] = ws.prof + words;
        }
    }
    if (trace && trace->start) {
        e = cudaEventRecord(trace->start, st);
        if (e != cudaSuccess) return e;
    }
    // full-slide mode: lane-owned items need 16-bit pair sums and a matrix
    // with a non-negative entry (full_desc_key's range); else one item per warp
    int8_t mmax = -128;
    for (int i = 0; i < kNSym * kNSym; i++) mmax = max(mmax, kp.m[i]);
    const bool full_lanes = kp.s.pair16 != 0 && mmax >= 0;
    for (int i = 0; i < nq; i++) {
        qs[i].items = reinterpret_cast<unsigned long long *>(ws.counters + (i == 0 ? kFullItems0 : kFullItems1));
        qs[i].status = d_status;
        size_t smem = (size_t)qs[i].smem_words * 4;
        const bool staged = qs[i].smem_words > 0;
        // length order: one CTA per SM, the widest whose profile(s) and slots fit
        const int wide = kp.s.mode != HS_MODE_FULL && staged && !input_order ? wide_warps(qs[i].smem_words) : 0;
        const ScanKernelFn kern = kp.s.mode == HS_MODE_FULL
                                      ? (full_lanes ? (staged ? scan_full_lanes_kernel<true> : scan_full_lanes_kernel<false>)
                                                    : (staged ? scan_full_kernel<true> : scan_full_kernel<false>))
                                      : wide ? pick_wide_kernel(wide, kp.s.pair16 != 0, share_steps)
                                             : pick_scan_kernel(staged, kp.s.pair16 != 0);
        if (wide) smem += wide * (kWarpSlotBytes + kHelpSlotBytes) + kCtaSlotBytes;
        const int threads = (kp.s.mode == HS_MODE_FULL ? kWarpsPerCta : wide ? wide : kScanWarps) * 32;
        int per_sm = 0;
        e = launch_fit(reinterpret_cast<const void *>(kern), threads, smem, &per_sm);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        // full-slide items: about four handed to each warp over the scan, so
        // that warps refill and balance (a flat step's units still fill all
        // 32 lanes)
        const bool full = kp.s.mode == HS_MODE_FULL;
        const int64_t work = (qs[i].end - qs[i].begin) * (full ? kp.s.rounds : 1);
        qs[i].lanes = lanes_for(work, (int64_t)per_sm * num_sms * (threads / 32) * (full ? 4 : 1));
        kern<<<per_sm * num_sms, threads, smem, st>>>(db, qs[i], srcs[i], kp.s, ws.scores, d_cells);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        nl++;
    }
    if (trace && trace->stop) {
        e = cudaEventRecord(trace->stop, st);
        if (e != cudaSuccess) return e;
    }
    if (launches) *launches += nl;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Batched scan: many queries against the resident database in one
// persistent launch.  Work items are (query, chunk) in query-major order;
// chunks are contiguous ranges of the length order with about equal
// residues, so the long targets of each query spread over many items.  A CTA
// takes an item, stages the query's profile for the role of the chunk's
// first (longest) target in shared memory -- only when the query or role
// changes -- and its warps run the pair loop over the chunk's positions from a
// CTA-shared counter.  Pairs of the other role (the one chunk per query that
// straddles the role switch) read that role's profile from global memory.
// ---------------------------------------------------------------------------
__global__ void chunk_bounds_kernel(const int64_t *cumres, int64_t n, int32_t nchunk, int64_t *bounds)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nchunk) return;
    const int64_t total = cumres[n];
    const int64_t target = (int64_t)((double)total * c / nchunk);
    int64_t lo = 0, hi = n;                 // first position whose cumulative residues reach target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cumres[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    bounds[c] = c == nchunk ? n : lo;
}

// Queries of one length class (their profiles share one shared-memory size)
// are listed by batch_classes_kernel; a scan launch covers one class.
struct BatchScan {
    int32_t nq, nchunk;
    const int32_t *qlist;           // the class's queries (batch indices)
    const unsigned *qcount;         // how many
    const int64_t *qoffsets;        // [nq + 1]
    const uint64_t *seeds;          // [nq]
    const int64_t *prof_off;        // [nq] word offsets into prof
    const uint32_t *prof;           // both role profiles of every query
    const int64_t *bounds;          // [nchunk + 1]
    int64_t long_end;
    int32_t *scores;                // [nq][n]
    unsigned *item_ctr;
    int64_t smem_words;             // profile words staged per CTA (wide kernel: slots follow)
    int32_t chunk_step;             // chunks per work item (wide CTAs take several)
};

// kSmem (length order): a chunk that straddles its query's role switch is run
// as two sub-ranges, each with its role's profile staged, so every profile
// read is a shared load.  Otherwise (database order, roles mixed) both role
// profiles are read from global memory.
// The batched scan's work loop, shared by the 8-warp kernel (slots in static
// shared memory) and the wide one (slots in dynamic shared memory after the
// profile).  prof_s: the staged role profile.
template <bool kSmem, bool P16>
__device__ __forceinline__ void batch_items(const DbView &db, const BatchScan &bs, const SParams &sp0,
                                            uint4 *prof_s, Plan *plans, FlatSlots *slots, long long &s_item,
                                            unsigned &s_pos)
{
    const uint32_t *prof_w = reinterpret_cast<const uint32_t *>(prof_s);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cur_q = -1, cur_role = -1;
    const int per_q = (bs.nchunk + bs.chunk_step - 1) / bs.chunk_step;     // items per query
    const long long nitems = (long long)*bs.qcount * per_q;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (long long)atomicAdd(bs.item_ctr, 1u);
            s_pos = 0;
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= nitems) break;
        const int ql = (int)(item / per_q), c = (int)(item - (long long)ql * per_q) * bs.chunk_step;
        const int q = bs.qlist[ql];
        const int64_t b0 = bs.bounds[c], b1 = bs.bounds[min(c + bs.chunk_step, bs.nchunk)];
        if (b0 < b1) {
            SParams sp = sp0;
            sp.qlen = (int32_t)(bs.qoffsets[q + 1] - bs.qoffsets[q]);
            sp.seed = bs.seeds[q];
            const int64_t words = profile_words(sp.qlen);
            const uint32_t *pg = bs.prof + bs.prof_off[q];
            QueryCtx qc;
            qc.scores = bs.scores + (int64_t)q * db.n;
            qc.cells = nullptr;
            if (kSmem) {
                // first position of the chunk whose target is shorter than the
                // query (targets are longest first)
                int64_t lo = b0, hi = b1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1, d = db.order[mid];
                    if (db.offsets[d + 1] - db.offsets[d] >= sp.qlen) lo = mid + 1;
                    else hi = mid;
                }
                for (int role = 0; role < 2; role++) {
                    const int64_t r0 = role ? lo : b0, r1 = role ? b1 : lo;
                    if (r0 >= r1) continue;
                    if (q != cur_q || role != cur_role) {
                        __syncthreads();                    // the previous profile is no longer read
                        const uint4 *src = reinterpret_cast<const uint4 *>(pg + (role ? words : 0));
                        for (int64_t i = threadIdx.x; i < words / 4; i += blockDim.x) prof_s[i] = src[i];
                        cur_q = q;
                        cur_role = role;
                    }
                    if (threadIdx.x == 0) s_pos = 0;
                    __syncthreads();
                    qc.prof_rev = prof_w;
                    qc.prof_fwd = prof_w;
                    const PosQueue pq = {r0, max(r0, min(bs.long_end, r1)), r1, &s_pos, 0xFFFFFFFFu};
                    run_pairs<P16>(db, sp, qc, pq, plans + 32 * w, slots + w, lane);
                    __syncthreads();                        // all warps are done with s_pos
                }
            } else {
                __syncthreads();
                qc.prof_rev = pg;
                qc.prof_fwd = pg + words;
                const PosQueue pq = {b0, max(b0, min(bs.long_end, b1)), b1, &s_pos, 0xFFFFFFFFu};
                run_pairs<P16>(db, sp, qc, pq, plans + 32 * w, slots + w, lane);
            }
        }
        __syncthreads();
    }
}

template <bool kSmem, bool P16>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 3)
scan_batch_kernel(DbView db, BatchScan bs, SParams sp0)
{
    extern __shared__ uint4 smem_raw[];
    __shared__ Plan plans[kWarpsPerCta * 32];
    __shared__ FlatSlots flat_slots[kWarpsPerCta];
    __shared__ long long s_item;
    __shared__ unsigned s_pos;
    batch_items<kSmem, P16>(db, bs, sp0, smem_raw, plans, flat_slots, s_item, s_pos);
}

// Long-query class: one CTA per SM of kWarps warps, the slots after the
// class's largest profile in dynamic shared memory.
template <bool P16, int kWarps>
__global__ void __launch_bounds__(kWarps * 32, 1)
scan_batch_wide_kernel(DbView db, BatchScan bs, SParams sp0)
{
    extern __shared__ uint4 smem_raw[];
    __shared__ long long s_item;
    __shared__ unsigned s_pos;
    Plan *plans = reinterpret_cast<Plan *>(smem_raw + bs.smem_words / 4);
    FlatSlots *slots = reinterpret_cast<FlatSlots *>(plans + kWarps * 32);
    batch_items<true, P16>(db, bs, sp0, smem_raw, plans, slots, s_item, s_pos);
}

typedef void (*BatchKernelFn)(DbView, BatchScan, SParams);

static BatchKernelFn pick_batch_wide_kernel(int warps, bool p16)
{
    if (warps == 24) return p16 ? scan_batch_wide_kernel<true, 24> : scan_batch_wide_kernel<false, 24>;
    return p16 ? scan_batch_wide_kernel<true, 12> : scan_batch_wide_kernel<false, 12>;
}

static BatchKernelFn pick_batch_kernel(bool smem, bool p16)
{
    if (smem) return p16 ? scan_batch_kernel<true, true> : scan_batch_kernel<true, false>;
    return p16 ? scan_batch_kernel<false, true> : scan_batch_kernel<false, false>;
}

// Splits the batch's queries into the length classes (qlen <= kBatchShortLen,
// and longer), in any order within a class.
__global__ void batch_classes_kernel(const int64_t *qoffsets, int32_t nq, int32_t *qlist, unsigned *counts)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const int c = qoffsets[q + 1] - qoffsets[q] <= kBatchShortLen ? 0 : 1;
        qlist[c * nq + atomicAdd(&counts[c], 1u)] = q;
    }
}

cudaError_t launch_scan_batch(const DbView &db, const int64_t *d_cumres, int64_t long_end, const KParams &kp,
                              const BatchLayout &bl, int32_t nchunk, int warps, int num_sms,
                              int32_t *d_status, cudaStream_t st, const ScanTrace *trace, int *launches,
                              bool input_order)
{
    ProfileJob job = {bl.queries, bl.qoffsets, bl.prof_off, 0, bl.prof, d_status};
    profile_kernel<<<dim3(16, bl.nq), 256, 0, st>>>(job, kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    chunk_bounds_kernel<<<(nchunk + 1 + 255) / 256, 256, 0, st>>>(d_cumres, db.n, nchunk, bl.bounds);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_classes_kernel<<<1, 256, 0, st>>>(bl.qoffsets, bl.nq, bl.qlist, bl.class_counts);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    BatchScan bs;
    bs.nq = bl.nq;
    bs.nchunk = nchunk;
    bs.qoffsets = bl.qoffsets;
    bs.seeds = bl.seeds;
    bs.prof_off = bl.prof_off;
    bs.prof = bl.prof;
    bs.bounds = bl.bounds;
    bs.long_end = long_end;
    bs.scores = bl.scores;
    const BatchKernelFn kern = pick_batch_kernel(!input_order, kp.s.pair16 != 0);
    if (trace && trace->start) {
        e = cudaEventRecord(trace->start, st);
        if (e != cudaSuccess) return e;
    }
    // one launch per length class, its shared memory sized for the class
    // (a class above the batch's longest query is known empty)
    int nl = 3;
    for (int c = 0; c < 2; c++) {
        if (c == 1 && bl.max_qlen <= kBatchShortLen) break;
        const int cls_len = c == 0 ? min(bl.max_qlen, kBatchShortLen) : bl.max_qlen;
        bs.qlist = bl.qlist + (int64_t)c * bl.nq;
        bs.qcount = bl.class_counts + c;
        bs.item_ctr = bl.item_ctrs + c;
        bs.smem_words = input_order ? 0 : profile_words(cls_len);
        size_t smem = (size_t)bs.smem_words * 4;
        // the widest CTA that fits the class's profile and slots, or the
        // tuning's choice of 24 or 12 warps when that fits
        int wide = !input_order ? wide_warps(bs.smem_words) : 0;
        if (wide && (warps == 12 || warps == 24) && warps < wide) wide = warps;
        bs.chunk_step = wide ? (wide + kWarpsPerCta - 1) / kWarpsPerCta : 1;
        const BatchKernelFn kc = wide ? pick_batch_wide_kernel(wide, kp.s.pair16 != 0) : kern;
        if (wide) smem += wide * kWarpSlotBytes;
        const int threads = (wide ? wide : kWarpsPerCta) * 32;
        int per_sm = 0;
        e = launch_fit(reinterpret_cast<const void *>(kc), threads, smem, &per_sm);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        kc<<<per_sm * num_sms, threads, smem, st>>>(db, bs, kp.s);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        nl++;
    }
    if (trace && trace->stop) {
        e = cudaEventRecord(trace->stop, st);
        if (e != cudaSuccess) return e;
    }
    if (launches) *launches += nl;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Replay of the ranked hits.  A CTA (or a warp) per hit reruns the pair with
// the same draws (so the scan itself never stores an alignment), checks the
// score against the scan's, and writes the winning round's run-length ops
// into the hit's slot.  The last CTA to finish packs the slots into the caller's ops
// buffer and fills in the offsets.  Batched: hit i belongs to query i / nhits.
// ---------------------------------------------------------------------------
struct ReplayArgs {
    const uint8_t *queries;         // letters (all queries when batched)
    const int64_t *qoffsets;        // nullptr: one query (sp.qlen, sp.seed)
    const uint64_t *seeds;          // batched: per query
    const int64_t *prof_off;        // batched: per query word offset into prof
    const uint32_t *prof;           // reversed profile, forward at + profile_words(qlen)
    const int64_t *hit_idx;         // nullptr: the single pair `single_index`
    int64_t single_index;
    const int32_t *hit_score;       // expected scores (nullptr: not checked)
    int32_t nhits;                  // hits per query
    int32_t k;                      // slot stride between queries, in hits
    int32_t nq;
    uint32_t *slots;                // (nq * k) * slot_stride
    int64_t slot_stride;
    int32_t *slot_len;
    hs_hit *hits;                   // nq * k records (query i at i * k)
    unsigned *ticket;               // nullptr: single pair, slots are the output
    uint32_t *ops;
    int64_t ops_cap;
    int64_t *ops_used;
    int32_t *status;
    int32_t stage;                  // kReplayStep: copy the hit's role profile into shared memory first
};

__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    atomicCAS(status, (int32_t)HS_OK, code);
}

// Three forms, each compiled alone (which keeps each kernel small):
// kReplayWarp, one warp per hit; kReplayStep, one CTA per hit of a one-round
// database-form search, all its warps scanning each step; kReplayRounds, one
// CTA of 24 warps per hit of a several-round search, its warps scoring the
// rounds in turn (one each up to 24 rounds) before warp 0 writes the best
// one's ops.
enum ReplayForm { kReplayWarp = 0, kReplayStep = 1, kReplayRounds = 2 };
constexpr int kReplayRoundWarps = 24;

template <int kForm> __host__ __device__ constexpr int replay_warps() { return kForm == kReplayRounds ? kReplayRoundWarps : kWarpsPerCta; }

template <int kForm>
__global__ void __launch_bounds__(replay_warps<kForm>() * 32) replay_kernel(DbView db, SParams sp0, ReplayArgs ra)
{
    constexpr int kW = replay_warps<kForm>();
    __shared__ int2 red[kW];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    constexpr bool cta = kForm != kReplayWarp;
    const int w = cta ? (int)blockIdx.x : (int)blockIdx.x * kW + warp;     // hit number over all queries
    const int per = max(ra.nhits, 1);
    const int qi = w / per, i = w - qi * per;
    if (ra.nhits > 0 && qi < ra.nq) {
        SParams sp = sp0;
        const uint32_t *prof = ra.prof;
        if (ra.qoffsets) {
            sp.qlen = (int32_t)(ra.qoffsets[qi + 1] - ra.qoffsets[qi]);
            sp.seed = ra.seeds[qi];
            prof += ra.prof_off[qi];
        }
        const int slot = qi * ra.k + i;
        const int64_t d = ra.hit_idx ? ra.hit_idx[slot] : ra.single_index;
        const int64_t off = db.offsets[d];
        PairCtx c;
        c.t = db.codes + off;
        c.tlen = (int32_t)(db.offsets[d + 1] - off);
        c.qlen = sp.qlen;
        c.qsmall = c.tlen >= sp.qlen;
        c.prof = prof + (c.qsmall ? 0 : profile_words(sp.qlen));
        c.S = profile_stride(sp.qlen);
        if constexpr (kForm == kReplayStep) {
            // a hit's steps run one after another, each reading profile
            // words: from shared memory they do not wait on L1/L2 misses
            if (ra.stage) {
                extern __shared__ uint4 rsm[];
                const int64_t n16 = profile_words(sp.qlen) / 4;
                const uint4 *src = reinterpret_cast<const uint4 *>(c.prof);
                for (int64_t x = threadIdx.x; x < n16; x += blockDim.x) rsm[x] = src[x];
                __syncthreads();
                c.prof = reinterpret_cast<const uint32_t *>(rsm);
            }
        }
        int64_t cells = 0;
        int br = 0;
        OpWriter ow;
        Span span = {-1, -1, -1, -1};
        ow.init(ra.slots + (int64_t)slot * ra.slot_stride, ra.slot_stride);
        int32_t best, again;
        if (ra.hit_score && ra.hit_score[slot] < sp.min_score) {
            best = again = ra.hit_score[slot];      // below the reporting threshold: no alignment
        } else if constexpr (kForm == kReplayStep) {
            // one round: it is the best one, and the scan's score checks the
            // replay; every warp scans each step, warp 0 writes the ops
            best = ra.hit_score[slot];
            again = align_round_cta<true>(c, sp, (uint64_t)d, 0, lane, warp, kW, red, cells, &ow, &span);
        } else if constexpr (kForm == kReplayRounds) {
            // warp w scores rounds w, w + kW, ...; the best (highest score,
            // then the first round, as AlignSequences keeps it) is run again
            // by warp 0, writing the ops
            int32_t wb = INT_MIN;
            int wr = INT_MAX;
            for (int r = warp; r < sp.rounds; r += kW) {
                const int32_t s = sp.mode == HS_MODE_FULL
                                      ? align_round_full<false>(c, sp, (uint64_t)d, r, lane, cells, nullptr, nullptr)
                                      : align_round<false>(c, sp, (uint64_t)d, r, lane, cells, nullptr, nullptr);
                if (s > wb) { wb = s; wr = r; }             // r ascends: the first best stays
            }
            if (lane == 0) red[warp] = make_int2(wb, wr);
            __syncthreads();
            best = INT_MIN;
            br = INT_MAX;
            for (int x = 0; x < kW; x++) {
                const int2 v = red[x];
                if (v.x > best || (v.x == best && v.y < br)) { best = v.x; br = v.y; }
            }
            again = best;
            if (warp == 0)
                again = sp.mode == HS_MODE_FULL ? align_round_full<true>(c, sp, (uint64_t)d, br, lane, cells, &ow, &span)
                                                : align_round<true>(c, sp, (uint64_t)d, br, lane, cells, &ow, &span);
        } else if (ra.hit_score && sp.rounds == 1) {
            best = ra.hit_score[slot];
            again = sp.mode == HS_MODE_FULL ? align_round_full<true>(c, sp, (uint64_t)d, 0, lane, cells, &ow, &span)
                                            : align_round<true>(c, sp, (uint64_t)d, 0, lane, cells, &ow, &span);
        } else {
            best = align_pair(c, sp, (uint64_t)d, lane, cells, &br);
            again = sp.mode == HS_MODE_FULL ? align_round_full<true>(c, sp, (uint64_t)d, br, lane, cells, &ow, &span)
                                            : align_round<true>(c, sp, (uint64_t)d, br, lane, cells, &ow, &span);
        }
        if (lane == 0 && (!cta || warp == 0)) {
            if (again != best || (ra.hit_score && ra.hit_score[slot] != best)) set_status(ra.status, HS_EINTERNAL);
            hs_hit h;
            h.db_index = d + sp.index_base;
            h.score = best;
            h.q_begin = span.qb; h.q_end = span.qe;
            h.t_begin = span.tb; h.t_end = span.te;
            h.ops_len = (int32_t)ow.n;
            h.ops_offset = 0;
            ra.hits[slot] = h;
            ra.slot_len[slot] = (int32_t)ow.n;
            if (!ra.ticket) {
                *ra.ops_used = ow.n;
                if (ow.n > ra.ops_cap) set_status(ra.status, HS_ETRUNC);
            }
        }
    }
    if (!ra.ticket) return;

    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ra.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // pack: offsets by an exclusive scan over all hits (one warp), then copy
    const int total_hits = ra.nq * ra.nhits;
    if (warp == 0) {
        int64_t carry = 0;
        for (int base = 0; base < total_hits; base += 32) {
            const int j = base + lane;
            const int slot = j < total_hits ? (j / ra.nhits) * ra.k + j % ra.nhits : 0;
            const int64_t v = j < total_hits ? ((volatile int32_t *)ra.slot_len)[slot] : 0;
            int64_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            if (j < total_hits) ((volatile int64_t *)&ra.hits[slot].ops_offset)[0] = carry + incl - v;
            carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        if (lane == 0) {
            *ra.ops_used = carry;
            if (carry > ra.ops_cap) set_status(ra.status, HS_ETRUNC);
        }
    }
    __syncthreads();
    for (int j = warp; j < total_hits; j += kW) {
        const int slot = (j / ra.nhits) * ra.k + j % ra.nhits;
        const int64_t o = ((volatile int64_t *)&ra.hits[slot].ops_offset)[0];
        const int32_t n = ((volatile int32_t *)ra.slot_len)[slot];
        if (o + n > ra.ops_cap) continue;
        const uint32_t *src = ra.slots + (int64_t)slot * ra.slot_stride;
        for (int x = lane; x < n; x += 32) ra.ops[o + x] = ((volatile const uint32_t *)src)[x];
    }
}

// One CTA per hit when its rounds or (one round, database form) its steps
// can be shared by the CTA's warps; one warp per hit otherwise.
// The one-round CTA form stages the hit's role profile in shared memory
// when one role of the longest query fits in 96 KB (queries up to ~1,000
// letters); in the 24-warp rounds form the copy loop cost 200 B of spills.
static void launch_replay_form(const DbView &db, const SParams &sp, const ReplayArgs &ra0, int64_t total,
                               int32_t max_qlen, cudaStream_t st)
{
    ReplayArgs ra = ra0;
    const size_t stage_bytes = (size_t)profile_words(max_qlen) * 4;
    ra.stage = stage_bytes <= 96 * 1024;
    const size_t smem = ra.stage ? stage_bytes : 0;
    int per_sm = 0;
    if (sp.rounds > 1) {
        ra.stage = 0;
        replay_kernel<kReplayRounds><<<(int)total, kReplayRoundWarps * 32, 0, st>>>(db, sp, ra);
    } else if (sp.mode == HS_MODE_DB && ra.hit_score) {
        if (ra.stage && launch_fit(reinterpret_cast<const void *>(replay_kernel<kReplayStep>), kWarpsPerCta * 32,
                                   smem, &per_sm) != cudaSuccess) ra.stage = 0;
        replay_kernel<kReplayStep><<<(int)total, kWarpsPerCta * 32, ra.stage ? smem : 0, st>>>(db, sp, ra);
    } else
        replay_kernel<kReplayWarp><<<(int)((total + kWarpsPerCta - 1) / kWarpsPerCta), kWarpsPerCta * 32, 0, st>>>(
            db, sp, ra);
}

static ReplayArgs replay_args_single(const uint8_t *d_query, const uint32_t *prof)
{
    ReplayArgs ra = {};
    ra.queries = d_query;
    ra.prof = prof;
    ra.nq = 1;
    return ra;
}

cudaError_t launch_replay(const DbView &db, const uint8_t *d_query, const KParams &kp,
                          const Workspace &ws, int32_t nhits, hs_hit *d_hits, uint32_t *d_ops,
                          int64_t ops_cap, int64_t *d_ops_used, int32_t *d_status, cudaStream_t st,
                          int *launches)
{
    if (nhits <= 0) return cudaSuccess;
    ReplayArgs ra = replay_args_single(d_query, ws.prof);
    ra.hit_idx = ws.hit_idx;
    ra.hit_score = ws.hit_score;
    ra.nhits = nhits;
    ra.k = nhits;
    ra.slots = ws.slots;
    ra.slot_stride = ws.slot_stride;
    ra.slot_len = ws.slot_len;
    ra.hits = d_hits;
    ra.ticket = ws.counters + kReplayTicket;
    ra.ops = d_ops;
    ra.ops_cap = ops_cap;
    ra.ops_used = d_ops_used;
    ra.status = d_status;
    launch_replay_form(db, kp.s, ra, nhits, kp.s.qlen, st);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_replay_batch(const DbView &db, const KParams &kp, const BatchLayout &bl, int32_t nhits,
                                int32_t k, hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap, int64_t *d_ops_used,
                                int32_t *d_status, cudaStream_t st, int *launches)
{
    if (nhits <= 0 || bl.nq <= 0) return cudaSuccess;
    ReplayArgs ra = replay_args_single(bl.queries, bl.prof);
    ra.qoffsets = bl.qoffsets;
    ra.seeds = bl.seeds;
    ra.prof_off = bl.prof_off;
    ra.hit_idx = bl.hit_idx;
    ra.hit_score = bl.hit_score;
    ra.nhits = nhits;
    ra.k = k;
    ra.nq = bl.nq;
    ra.slots = bl.slots;
    ra.slot_stride = bl.slot_stride;
    ra.slot_len = bl.slot_len;
    ra.hits = d_hits;
    ra.ticket = bl.replay_ticket;
    ra.ops = d_ops;
    ra.ops_cap = ops_cap;
    ra.ops_used = d_ops_used;
    ra.status = d_status;
    const int64_t total = (int64_t)bl.nq * nhits;
    launch_replay_form(db, kp.s, ra, total, bl.max_qlen, st);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// hs_get_alignment: the profile kernel, then one warp writing straight into
// the caller's ops buffer.  `ws` supplies the profile.
cudaError_t launch_replay_one(const DbView &db, const uint8_t *d_query, const KParams &kp,
                              const Workspace &ws, int64_t db_index, uint32_t *d_ops, int64_t cap,
                              hs_hit *d_hit, int64_t *d_ops_used, int32_t *d_status, cudaStream_t st)
{
    ProfileJob job = {d_query, nullptr, nullptr, kp.s.qlen, ws.prof, d_status};
    profile_kernel<<<64, 256, 0, st>>>(job, kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ReplayArgs ra = replay_args_single(d_query, ws.prof);
    ra.hit_idx = nullptr;
    ra.single_index = db_index;
    ra.nhits = 1;
    ra.k = 1;
    ra.slots = d_ops;
    ra.slot_stride = cap;
    ra.slot_len = ws.slot_len;
    ra.hits = d_hit;
    ra.ticket = nullptr;
    ra.ops = d_ops;
    ra.ops_cap = cap;
    ra.ops_used = d_ops_used;
    ra.status = d_status;
    launch_replay_form(db, kp.s, ra, 1, kp.s.qlen, st);
    return cudaGetLastError();
}

}  // namespace hs
