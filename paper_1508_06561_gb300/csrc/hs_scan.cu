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
    const int S = profile_stride(kp.qlen);
    const int64_t words = profile_words(kp.qlen);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < 2 * words;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const bool rev = idx < words;
        const int64_t i = rev ? idx : idx - words;
        const int r = (int)(i / (kNSym * S));
        const int rem = (int)(i - (int64_t)r * kNSym * S);
        const int a = rem / S, w = rem - a * S;
        prof[idx] = profile_word_value(q, kp.qlen, rev, msm, kp.bias, r, a, w);
    }
}

// ---------------------------------------------------------------------------
// The scan.  A persistent grid; each warp repeatedly takes work from a queue
// over the length-ordered database (longest first): targets of at least
// kLongLen letters one at a time, the rest kShortChunk at a time.  Every
// pair writes only its score (and, if asked, its cell count).
// ---------------------------------------------------------------------------
struct ScanRange {
    int64_t begin, long_end, end;   // sorted positions [begin, end); [begin, long_end) long
    uint32_t *ctr_long, *ctr_short;
    int qsmall;                     // role shared by every pair of the range
    int prof_off;                   // word offset of this role's profile in shared memory
};

// Up to two ranges (the two roles).  With both profiles resident, one launch
// drains the long-target range first and then the short one, so the whole
// database is a single longest-first queue.
struct ScanPlan {
    ScanRange rg[2];
    int nranges;
    int64_t smem_words;             // profile words to copy from prof_g
};

__global__ void __launch_bounds__(kWarpsPerCta * 32, 4)
scan_kernel(DbView db, ScanPlan plan, const uint32_t *__restrict__ prof_g, KParams kp,
            int32_t *__restrict__ scores, int64_t *__restrict__ cells_out)
{
    extern __shared__ uint4 smem_raw[];
    uint32_t *prof = reinterpret_cast<uint32_t *>(smem_raw);
    const int S = profile_stride(kp.qlen);
    {
        const int64_t n16 = plan.smem_words / 4;   // profile words are a multiple of 4
        const uint4 *src = reinterpret_cast<const uint4 *>(prof_g);
        for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) smem_raw[i] = src[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    for (int ri = 0; ri < plan.nranges; ri++) {
        const ScanRange rg = ri == 0 ? plan.rg[0] : plan.rg[1];   // no dynamic param indexing
        int long_done = rg.long_end <= rg.begin;
        for (;;) {
            int64_t start = 0, cnt = 0;
            if (lane == 0) {
                if (!long_done) {
                    const int64_t i = rg.begin + (int64_t)atomicAdd(rg.ctr_long, 1u);
                    if (i < rg.long_end) { start = i; cnt = 1; }
                    else long_done = 1;
                }
                if (cnt == 0) {
                    start = max(rg.long_end, rg.begin) + (int64_t)atomicAdd(rg.ctr_short, (uint32_t)kShortChunk);
                    cnt = min((int64_t)kShortChunk, rg.end - start);
                }
            }
            start = __shfl_sync(0xFFFFFFFFu, start, 0);
            cnt = __shfl_sync(0xFFFFFFFFu, cnt, 0);
            long_done = __shfl_sync(0xFFFFFFFFu, long_done, 0);
            if (cnt <= 0) break;
            for (int64_t pos = start; pos < start + cnt; pos++) {
                const int64_t d = db.order[pos];
                const int64_t off = db.offsets[d];
                PairCtx c;
                c.prof = prof + rg.prof_off;
                c.S = S;
                c.t = db.codes + off;
                c.tlen = (int32_t)(db.offsets[d + 1] - off);
                c.qlen = kp.qlen;
                c.qsmall = rg.qsmall != 0;
                int64_t cells = 0;
                const int32_t s = align_pair(c, kp, (uint64_t)d, lane, cells, nullptr);
                if (lane == 0) {
                    scores[d] = s;
                    if (cells_out) cells_out[d] = cells;
                }
            }
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

    ScanRange r[2];
    for (int role = 0; role < 2; role++) {
        ScanRange &rg = r[role];
        rg.qsmall = role == 0;
        rg.begin = role == 0 ? 0 : split;
        rg.end = role == 0 ? split : db.n;
        rg.long_end = role == 0 ? min(long_end, split) : rg.begin;
        rg.ctr_long = ws.counters + (role == 0 ? kQsLong : kQlLong);
        rg.ctr_short = ws.counters + (role == 0 ? kQsShort : kQlShort);
        rg.prof_off = 0;
    }
    const bool fused = fuse_roles(kp.qlen);
    ScanPlan plans[2];
    const uint32_t *srcs[2];
    int nplans = 0;
    if (fused) {
        ScanPlan &pl = plans[nplans];
        pl.nranges = 0;
        for (int role = 0; role < 2; role++) {
            if (r[role].end <= r[role].begin) continue;
            r[role].prof_off = role == 0 ? 0 : (int)words;
            pl.rg[pl.nranges++] = r[role];
        }
        pl.smem_words = 2 * words;
        srcs[nplans] = ws.prof;
        if (pl.nranges) nplans++;
    } else {
        for (int role = 0; role < 2; role++) {
            if (r[role].end <= r[role].begin) continue;
            ScanPlan &pl = plans[nplans];
            pl.rg[0] = r[role];
            pl.nranges = 1;
            pl.smem_words = words;
            srcs[nplans] = ws.prof + (role == 0 ? 0 : words);
            nplans++;
        }
    }
    if (trace && trace->start) {
        e = cudaEventRecord(trace->start, st);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < nplans; i++) {
        const size_t smem = (size_t)plans[i].smem_words * 4;
        e = cudaFuncSetAttribute(scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel, kWarpsPerCta * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        scan_kernel<<<per_sm * num_sms, kWarpsPerCta * 32, smem, st>>>(db, plans[i], srcs[i], kp, ws.scores,
                                                                        d_cells);
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
