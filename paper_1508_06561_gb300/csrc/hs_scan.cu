// hs_scan.cu -- the database scan (every pair's score) and the alignment
// replay of the ranked hits.  Database-search form of Fig. 1 (Sec. III.B.3).
#include <cuda_runtime.h>

#include "hs_device.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// Profile preparation: both role profiles (reversed and forward query) into
// global memory, once per search; the scan CTAs copy theirs into shared
// memory and the replay reads them in place.
// ---------------------------------------------------------------------------
__global__ void profile_kernel(const uint8_t *__restrict__ q, KParams kp, uint32_t *__restrict__ prof)
{
    __shared__ int8_t msm[kNSym * kNSym];
    for (int i = threadIdx.x; i < kNSym * kNSym; i += blockDim.x) msm[i] = kp.m[i];
    __syncthreads();
    const int R = profile_stride(kp.qlen);
    const int64_t words = profile_words(kp.qlen);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * words;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const bool rev = idx < words;
        const int64_t i = rev ? idx : idx - words;
        const int a = (int)(i / R), s = (int)(i - (int64_t)a * R);
        prof[idx] = profile_word_value(q, kp.qlen, rev, msm, kp.bias, a, s);
    }
}

// ---------------------------------------------------------------------------
// The scan.  A persistent grid over one queue of length-ordered database
// positions (longest first).  Every lane of a warp owns one pair: its O(1)
// state (Sec. III.B.4) -- positions, step, score, best round, size factors,
// one cached Philox block -- sits in that lane's registers, so the step
// bookkeeping of 32 pairs runs as one SIMT instruction stream.  Each round of
// the loop plans one step for every held pair.  Small steps (at most
// kLocalIters chunk iterations) are scored by their own lane; the others one
// at a time by the whole warp (coop_scan), reading the step's plan from the
// warp's shared-memory plan slots.  Targets of >= kLongLen letters are taken
// one per warp (only lane 0 holds a pair) so each gets the warp alone.
// ---------------------------------------------------------------------------
constexpr int kLocalIters = 64;

struct ScanQueue {
    int64_t begin, long_end, end;   // sorted positions [begin, end); [begin, long_end) long
    uint32_t *ctr;
    int64_t smem_words;             // profile words staged into shared memory
    int rev_off, fwd_off;           // word offsets of the two role profiles (-1: absent)
};

struct Lane {                       // one pair held by one lane
    int64_t d;                      // database index, -1 = empty
    const uint8_t *t;
    int32_t nl, ns, qsmall;
    int32_t Lp, Sp, step, score, best, round;
    uint32_t lf, sf;
    int64_t cells;
    int64_t blk;                    // Philox block cached in w0..w3
    uint64_t w0, w1, w2, w3;
};

__device__ __forceinline__ uint32_t lane_draw(Lane &L, const KParams &kp, uint64_t i)
{
    const int64_t b = (int64_t)(i >> 4);
    if (b != L.blk) {
        uint64_t o[4];
        philox4x64_10((uint64_t)L.d, (uint64_t)L.round, (uint64_t)b, 0, kp.seed, 0, o);
        L.w0 = o[0]; L.w1 = o[1]; L.w2 = o[2]; L.w3 = o[3];
        L.blk = b;
    }
    const unsigned wi = (unsigned)(i >> 2) & 3u;
    const uint64_t w = wi == 0 ? L.w0 : wi == 1 ? L.w1 : wi == 2 ? L.w2 : L.w3;
    return (uint32_t)(w >> (48 - 16 * (unsigned)(i & 3))) & 0xFFFFu;
}

// Start round L.round: lf = MAX(minFactor, LFactor*random()), sf likewise.
__device__ __forceinline__ void lane_start_round(Lane &L, const KParams &kp)
{
    L.blk = -1;
    uint32_t lf = (uint32_t)(((uint64_t)kp.lf_q16 * lane_draw(L, kp, 0)) >> 16);
    uint32_t sf = (uint32_t)(((uint64_t)kp.sf_q16 * lane_draw(L, kp, 1)) >> 16);
    L.lf = max(lf, kp.minf_q16);
    L.sf = max(sf, kp.minf_q16);
    L.Lp = 0; L.Sp = 0; L.step = 0; L.score = 0;
}

// Finish every round whose loop has ended (Fig. 1: "append the remaining
// with dashes"; AlignSequences keeps the first best round), then the pair.
__device__ __forceinline__ void lane_settle(Lane &L, const KParams &kp, int32_t *scores, int64_t *cells_out)
{
    while (L.d >= 0 && !(L.Lp < L.nl && L.Sp < L.ns)) {
        L.score -= kp.pgp * ((L.nl - L.Lp) + (L.ns - L.Sp));
        if (L.score > L.best) L.best = L.score;
        L.round++;
        if (L.round < kp.rounds) {
            lane_start_round(L, kp);
        } else {
            scores[L.d] = L.best;
            if (cells_out) cells_out[L.d] = L.cells;
            L.d = -1;
        }
    }
}

__global__ void __launch_bounds__(kWarpsPerCta * 32, 3)
scan_kernel(DbView db, ScanQueue qu, const uint32_t *__restrict__ prof_g, KParams kp,
            int32_t *__restrict__ scores, int64_t *__restrict__ cells_out)
{
    extern __shared__ uint4 smem_raw[];
    __shared__ Plan plans[kWarpsPerCta][32];
    const uint32_t *prof = reinterpret_cast<const uint32_t *>(smem_raw);
    const int S = profile_stride(kp.qlen);
    {
        const int64_t n16 = qu.smem_words / 4;          // profile words are a multiple of 4
        const uint4 *src = reinterpret_cast<const uint4 *>(prof_g);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) smem_raw[i] = src[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    Lane L = {};
    L.d = -1;
    L.t = db.codes;
    L.best = INT_MIN;
    int phase = qu.long_end > qu.begin ? 0 : 1;       // 0: one long target per warp
    bool open = true;
    for (;;) {
        // refill empty lanes from the queue
        if (open) {
            unsigned need = __ballot_sync(0xFFFFFFFFu, L.d < 0);
            if (phase == 0) need &= 1u;
            if (need) {
                const int m = __popc(need);
                long long base = 0;
                if (lane == 0) base = (long long)qu.begin + (long long)atomicAdd(qu.ctr, (uint32_t)m);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (base + m >= qu.end) open = false;
                if (phase == 0 && base >= qu.long_end) phase = 1;
                const long long pos = base + __popc(need & lt_mask);
                if (((need >> lane) & 1u) && pos < qu.end) {
                    L.d = db.order[pos];
                    const int64_t off = db.offsets[L.d];
                    const int32_t tlen = (int32_t)(db.offsets[L.d + 1] - off);
                    L.t = db.codes + off;
                    L.qsmall = tlen >= kp.qlen;            // the target is large on ties
                    L.nl = L.qsmall ? tlen : kp.qlen;
                    L.ns = L.qsmall ? kp.qlen : tlen;
                    L.round = 0;
                    L.best = INT_MIN;
                    L.cells = 0;
                    lane_start_round(L, kp);
                    lane_settle(L, kp, scores, cells_out);   // empty small sequence
                }
            }
        }
        __syncwarp();
        const bool busy = L.d >= 0;
        if (!open && __ballot_sync(0xFFFFFFFFu, busy) == 0) break;

        // plan one step per held pair (Fig. 1's Align: ls and ss, A6)
        Plan g = {L.t, L.Lp, L.Sp, 1, 1, L.qsmall, 0, 0, 0};
        int32_t vmax = 0, kstar = 0;
        bool local = false;
        if (busy) {
            const int32_t Lrem = L.nl - L.Lp, Srem = L.ns - L.Sp;
            const int32_t ls = max((int32_t)(((uint64_t)Lrem * L.lf) >> 16), 1);
            const uint64_t u = lane_draw(L, kp, 2 + (uint64_t)L.step);
            const int64_t ssw = (int64_t)(((uint64_t)Srem * L.sf * u) >> 32);
            g.ls = ls;
            g.ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)min(Srem, ls)));
            const int64_t iters = (int64_t)((ls - g.ss + 4) >> 2) * (g.ss + (L.qsmall ? 3 : 0));
            local = iters <= kLocalIters;
            if (local) {
                lane_scan(prof + (L.qsmall ? qu.rev_off : qu.fwd_off), S, kp.qlen, g, kp.bias, kp.flush,
                          vmax, kstar);
            } else {
                plan_grid(g);
                plans[threadIdx.x >> 5][lane] = g;
            }
        }
        __syncwarp();
        // the other steps, one pair at a time, by the whole warp
        unsigned coop = __ballot_sync(0xFFFFFFFFu, busy && !local);
        while (coop) {
            const int i = __ffs(coop) - 1;
            coop &= coop - 1;
            const Plan h = plans[threadIdx.x >> 5][i];
            int32_t v, k;
            coop_scan(prof + (h.qsmall ? qu.rev_off : qu.fwd_off), S, kp.qlen, h, kp.bias, kp.flush, lane, v, k);
            if (lane == i) { vmax = v; kstar = k; }
        }
        // consume (Fig. 1: delete the used-up parts) and score incrementally (A17)
        if (busy) {
            L.cells += (int64_t)(g.ls - g.ss + 1) * g.ss;
            int32_t gap = 0;
            if (kstar > 0) gap = (L.step == 0) ? kp.pgp * kstar : kp.gop + (kstar - 1) * kp.gep;
            L.score += vmax - gap;
            L.Lp += kstar + g.ss;
            L.Sp += g.ss;
            L.step++;
            lane_settle(L, kp, scores, cells_out);
        }
    }
}

size_t scan_smem_bytes(int32_t qlen) { return (size_t)profile_words(qlen) * 4; }

// Both profiles share one launch when they fit twice per SM with room to spare.
static bool fuse_roles(int32_t qlen) { return 2 * scan_smem_bytes(qlen) <= 100 * 1024; }

cudaError_t launch_scan(const DbView &db, int64_t split, int64_t long_end, const uint8_t *d_query,
                        const KParams &kp, const Workspace &ws, int64_t *d_cells, int num_sms,
                        cudaStream_t st, const ScanTrace *trace, int *launches)
{
    const int64_t words = profile_words(kp.qlen);
    profile_kernel<<<64, 256, 0, st>>>(d_query, kp, ws.prof);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int nl = 1;

    ScanQueue qs[2];
    const uint32_t *srcs[2];
    int nq = 0;
    if (fuse_roles(kp.qlen)) {
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
            q.smem_words = words; q.rev_off = 0; q.fwd_off = -1;
            srcs[nq++] = ws.prof;
        }
        if (split < db.n) {
            ScanQueue &q = qs[nq];
            q.begin = split; q.end = db.n; q.long_end = split;   // every target is shorter than the query
            q.ctr = ws.counters + kQlLong;
            q.smem_words = words; q.rev_off = -1; q.fwd_off = 0;
            srcs[nq++] = ws.prof + words;
        }
    }
    if (trace && trace->start) {
        e = cudaEventRecord(trace->start, st);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < nq; i++) {
        const size_t smem = (size_t)qs[i].smem_words * 4;
        e = cudaFuncSetAttribute(scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel, kWarpsPerCta * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        scan_kernel<<<per_sm * num_sms, kWarpsPerCta * 32, smem, st>>>(db, qs[i], srcs[i], kp, ws.scores, d_cells);
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
// Replay of the ranked hits.  One warp per hit reruns the pair with the same
// draws (so the scan itself never stores an alignment), checks the score
// against the scan's, and writes the winning round's run-length ops into the
// hit's slot.  The last CTA to finish packs the slots into the caller's ops
// buffer and fills in the offsets.
// ---------------------------------------------------------------------------
struct ReplayArgs {
    const uint32_t *prof;           // reversed profile, forward at + words
    int64_t words;
    const int64_t *hit_idx;         // nullptr: the single pair `single_index`
    int64_t single_index;
    const int32_t *hit_score;       // expected scores (nullptr: not checked)
    int32_t nhits;
    uint32_t *slots;                // nhits * slot_stride
    int64_t slot_stride;
    int32_t *slot_len;
    hs_hit *hits;
    uint32_t *ticket;               // nullptr: single pair, slots are the output
    uint32_t *ops;
    int64_t ops_cap;
    int64_t *ops_used;
    int32_t *status;
};

__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    atomicCAS(status, (int32_t)HS_OK, code);
}

__global__ void __launch_bounds__(kWarpsPerCta * 32) replay_kernel(DbView db, KParams kp, ReplayArgs ra)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kWarpsPerCta + warp;
    if (i < ra.nhits) {
        const int64_t d = ra.hit_idx ? ra.hit_idx[i] : ra.single_index;
        const int64_t off = db.offsets[d];
        PairCtx c;
        c.t = db.codes + off;
        c.tlen = (int32_t)(db.offsets[d + 1] - off);
        c.qlen = kp.qlen;
        c.qsmall = c.tlen >= kp.qlen;
        c.prof = ra.prof + (c.qsmall ? 0 : ra.words);
        c.S = profile_stride(kp.qlen);
        int64_t cells = 0;
        int br = 0;
        const int32_t best = align_pair(c, kp, (uint64_t)d, lane, cells, &br);
        OpWriter ow;
        Span span = {-1, -1, -1, -1};
        ow.init(ra.slots + (int64_t)i * ra.slot_stride, ra.slot_stride);
        const int32_t again = align_round<true>(c, kp, (uint64_t)d, br, lane, cells, &ow, &span);
        if (lane == 0) {
            if (again != best || (ra.hit_score && ra.hit_score[i] != best)) set_status(ra.status, HS_EINTERNAL);
            hs_hit h;
            h.db_index = d;
            h.score = best;
            h.q_begin = span.qb; h.q_end = span.qe;
            h.t_begin = span.tb; h.t_end = span.te;
            h.ops_len = (int32_t)ow.n;
            h.ops_offset = 0;
            ra.hits[i] = h;
            ra.slot_len[i] = (int32_t)ow.n;
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

    // pack: offsets by an exclusive scan over the hits (one warp), then copy
    if (warp == 0) {
        int64_t carry = 0;
        for (int base = 0; base < ra.nhits; base += 32) {
            const int j = base + lane;
            int64_t v = j < ra.nhits ? ((volatile int32_t *)ra.slot_len)[j] : 0;
            int64_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            if (j < ra.nhits) ((volatile int64_t *)&ra.hits[j].ops_offset)[0] = carry + incl - v;
            carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        if (lane == 0) {
            *ra.ops_used = carry;
            if (carry > ra.ops_cap) set_status(ra.status, HS_ETRUNC);
        }
    }
    __syncthreads();
    __threadfence_block();
    for (int j = warp; j < ra.nhits; j += kWarpsPerCta) {
        const int64_t o = ((volatile int64_t *)&ra.hits[j].ops_offset)[0];
        const int32_t n = ((volatile int32_t *)ra.slot_len)[j];
        if (o + n > ra.ops_cap) continue;
        const uint32_t *src = ra.slots + (int64_t)j * ra.slot_stride;
        for (int x = lane; x < n; x += 32) ra.ops[o + x] = ((volatile const uint32_t *)src)[x];
    }
}

cudaError_t launch_replay(const DbView &db, const uint8_t *d_query, const KParams &kp,
                          const Workspace &ws, int32_t nhits, hs_hit *d_hits, uint32_t *d_ops,
                          int64_t ops_cap, int64_t *d_ops_used, int32_t *d_status, cudaStream_t st,
                          int *launches)
{
    (void)d_query;
    if (nhits <= 0) return cudaSuccess;
    ReplayArgs ra;
    ra.prof = ws.prof;
    ra.words = profile_words(kp.qlen);
    ra.hit_idx = ws.hit_idx;
    ra.single_index = 0;
    ra.hit_score = ws.hit_score;
    ra.nhits = nhits;
    ra.slots = ws.slots;
    ra.slot_stride = ws.slot_stride;
    ra.slot_len = ws.slot_len;
    ra.hits = d_hits;
    ra.ticket = ws.counters + kReplayTicket;
    ra.ops = d_ops;
    ra.ops_cap = ops_cap;
    ra.ops_used = d_ops_used;
    ra.status = d_status;
    const int grid = (nhits + kWarpsPerCta - 1) / kWarpsPerCta;
    replay_kernel<<<grid, kWarpsPerCta * 32, 0, st>>>(db, kp, ra);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// hs_get_alignment: the profile kernel, then one warp writing straight into
// the caller's ops buffer.  `ws` supplies the profile and one hit slot.
cudaError_t launch_replay_one(const DbView &db, const uint8_t *d_query, const KParams &kp,
                              const Workspace &ws, int64_t db_index, uint32_t *d_ops, int64_t cap,
                              hs_hit *d_hit, int64_t *d_ops_used, int32_t *d_status, cudaStream_t st)
{
    profile_kernel<<<64, 256, 0, st>>>(d_query, kp, ws.prof);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ReplayArgs ra;
    ra.prof = ws.prof;
    ra.words = profile_words(kp.qlen);
    ra.hit_idx = nullptr;
    ra.single_index = db_index;
    ra.hit_score = nullptr;
    ra.nhits = 1;
    ra.slots = d_ops;
    ra.slot_stride = cap;
    ra.slot_len = ws.slot_len;
    ra.hits = d_hit;
    ra.ticket = nullptr;
    ra.ops = d_ops;
    ra.ops_cap = cap;
    ra.ops_used = d_ops_used;
    ra.status = d_status;
    replay_kernel<<<1, kWarpsPerCta * 32, 0, st>>>(db, kp, ra);
    return cudaGetLastError();
}

}  // namespace hs
