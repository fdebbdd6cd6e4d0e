// hs_internal.h -- declarations shared by the library's translation units
// (host runtime <-> kernels).  Not part of the public C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "hsearch.h"

namespace hs {

constexpr int kNSym = 24;               // BLOSUM62 alphabet (Sec. III.A)
constexpr int kWarpsPerCta = 8;         // scan kernel: 256 threads
constexpr int kTopkThreads = 512;
constexpr int kLongLen = 2048;          // targets this long are scheduled one per warp
constexpr int kShortChunk = 8;          // shorter targets are taken 8 at a time
constexpr int kCodesPad = 64;           // readable bytes past the last residue

// Query profile geometry: for each of the 24 letters a row of R words,
// word s packing the biased scores of stored columns s..s+3 (4 zero columns
// before the query, 12 after).  R is odd, so the 24 rows of one column fall
// in 24 distinct shared-memory banks.
__host__ __device__ inline int profile_stride(int qlen) { return (qlen + 16) | 1; }
__host__ __device__ inline int64_t profile_words(int qlen) { return (int64_t)kNSym * profile_stride(qlen); }

// What the scan and replay need to score pairs of one query; passed by
// value as kernel arguments, so launching needs no parameter copies.
struct SParams {
    int32_t bias;                       // -min(M): M + bias >= 0
    int32_t flush;                      // byte-lane flush interval: floor(255 / (max-min))
    int32_t pgp, gop, gep, rounds;
    uint32_t lf_q16, sf_q16, minf_q16;  // LFactor, SFactor, MinFactor in Q16
    int32_t qlen;
    uint64_t seed;
    int64_t index_base;                 // database index of the first loaded sequence (shards)
    int32_t min_score;                  // replay only hits scoring >= this (threshold search)
    int32_t mode;                       // HS_MODE_DB or HS_MODE_FULL
    int32_t pair16;                     // 16-bit chunk sums suffice: (max-min) * (qlen+3) <= 65535
    int32_t pack_shifts;                // cell counts also carry the shifts scanned, << 40 (profiling)
    int32_t flat_min_chunks;            // a step joins the flat unit list with at least this many 4-shift
    int32_t flat_max_iters;             // chunks, or at most this many iterations per chunk (else lane grid)
    int32_t help_min_units;             // a warp's lone flat step of at least this many units is shared
};                                      // with its CTA's idle warps (the scan_wide_kernel launches)
constexpr int kFlatMinChunks = 16;      // defaults of the two (a tuning may change them)
constexpr int kFlatMaxIters = 128;
constexpr int kHelpMinUnits = 256;
constexpr int kHelpLen = 8192;

// The matrix (for building profiles) plus the scoring parameters.
struct KParams {
    int8_t m[kNSym * kNSym];            // M[query letter][target letter]
    SParams s;
};

// Device view of a loaded database.
struct DbView {
    const uint8_t *codes;               // residues, kCodesPad readable bytes past the end
    const int64_t *offsets;             // n + 1
    const int32_t *order;               // database indices, longest first
    int64_t n;
};

// Workspace carve-up (all offsets 256-byte aligned).
struct Workspace {
    uint32_t *prof;                     // [2 * profile words] reversed, then forward query profile
    int32_t *scores;                    // [n] by database index
    uint32_t *counters;                 // [kNumCounters], zeroed per search
    uint64_t *cand;                     // [topk_ctas * k] per-CTA top-k keys
    int64_t *hit_idx;                   // [k] database index of each ranked hit
    int32_t *hit_score;                 // [k]
    uint32_t *slots;                    // [k * slot_stride] replayed ops
    int32_t *slot_len;                  // [k]
    int64_t slot_stride;
    int32_t topk_ctas;
    int32_t k;
};
// kFullItems0/1: 64-bit item counters (two words each) of the full-slide
// scan's one or two queues, at 8-byte aligned offsets.
enum Counter { kQsLong = 0, kQsShort = 1, kQlLong = 2, kQlShort = 3, kTopkTicket = 4, kReplayTicket = 5,
               kFullItems0 = 8, kFullItems1 = 10, kNumCounters = 12 };

constexpr int kTopkCtas = 152;

// Device layout of a batched search (many queries, one scan launch).
struct BatchLayout {
    int32_t nq, max_qlen;
    const uint8_t *queries;             // letters of all queries
    const int64_t *qoffsets;            // [nq + 1]
    const uint64_t *seeds;              // [nq]
    int64_t *prof_off;                  // [nq] word offset of each query's two profiles
    uint32_t *prof;                     // profiles of every query
    int64_t *bounds;                    // [nchunk + 1] chunk boundaries in the length order
    int32_t *scores;                    // [nq][n]
    unsigned *counters;                 // item counters and query counts of the two length classes,
                                        // replay ticket, then one top-k ticket per query
    unsigned *item_ctrs, *class_counts, *replay_ticket, *topk_tickets;
    int32_t *qlist;                     // [2][nq] queries of each length class
    uint64_t *cand;                     // [nq][kTopkCtas * k]
    int64_t *hit_idx;                   // [nq * k]
    int32_t *hit_score;                 // [nq * k]
    uint32_t *slots;                    // [nq * k][slot_stride]
    int64_t slot_stride;
    int32_t *slot_len;                  // [nq * k]
    int64_t counter_bytes;
};
constexpr int kMaxChunks = 8192;
constexpr int kBatchShortLen = 512;     // batched scan: queries up to this long form the short class
constexpr int kDefaultChunks = 1024;

// The scan schedule (hs_sort.cu): d_order = database indices longest first
// (ties in database order) or in database order; d_sorted_len = their
// lengths; d_cumres[i] = residues before schedule position i (n + 1).
size_t schedule_scratch_bytes(int64_t n);
cudaError_t build_schedule(const int64_t *d_offsets, int64_t n, int32_t maxlen, bool by_length, int32_t *d_order,
                           int64_t *d_cumres, int32_t *d_sorted_len, void *d_scratch, cudaStream_t st);

size_t workspace_bytes(int64_t n, int32_t qlen, int32_t k);
Workspace carve_workspace(void *base, int64_t n, int32_t qlen, int32_t k);
int64_t slot_stride_for(int32_t qlen);

// Launchers (hs_scan.cu / hs_topk.cu).  Return a cudaError_t.
// Role split: targets at sorted positions [0, split) are at least as long
// as the query (the query is the small sequence); [split, n) are shorter.
// long_end: sorted positions [0, long_end) hold targets of >= kLongLen letters.
// trace (optional): events recorded around the scan launch(es).
// launches (optional): incremented by the number of kernels launched.
// share_steps: the wide scan's warps share large lone steps at the scan's
// end (the caller sets it for databases with at least one target of
// kHelpLen letters or more per SM).
struct ScanTrace {
    cudaEvent_t start, stop;
};
cudaError_t launch_scan(const DbView &db, int64_t split, int64_t long_end, const uint8_t *d_query,
                        const KParams &kp, const Workspace &ws, int64_t *d_cells, int32_t *d_status, int num_sms,
                        cudaStream_t st, const ScanTrace *trace, int *launches, bool input_order,
                        bool share_steps);
size_t scan_smem_bytes(int32_t qlen);
cudaError_t launch_topk(const Workspace &ws, int64_t n, int32_t k, cudaStream_t st, int *launches);
cudaError_t launch_topk_batch(const BatchLayout &bl, int64_t n, int32_t k, int32_t nhits, cudaStream_t st,
                              int *launches);
cudaError_t launch_prof_offsets(const BatchLayout &bl, cudaStream_t st);
cudaError_t launch_scan_batch(const DbView &db, const int64_t *d_cumres, int64_t long_end, const KParams &kp,
                              const BatchLayout &bl, int32_t nchunk, int warps, int num_sms,
                              int32_t *d_status, cudaStream_t st, const ScanTrace *trace, int *launches,
                              bool input_order);
cudaError_t launch_replay_batch(const DbView &db, const KParams &kp, const BatchLayout &bl, int32_t nhits,
                                int32_t k, hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap, int64_t *d_ops_used,
                                int32_t *d_status, cudaStream_t st, int *launches);
cudaError_t launch_count_at_least(const int32_t *scores, int64_t n, int32_t threshold, int64_t *d_count,
                                  int num_sms, cudaStream_t st, int *launches);
cudaError_t launch_replay(const DbView &db, const uint8_t *d_query, const KParams &kp,
                          const Workspace &ws, int32_t nhits, hs_hit *d_hits, uint32_t *d_ops,
                          int64_t ops_cap, int64_t *d_ops_used, int32_t *d_status, cudaStream_t st,
                          int *launches);
cudaError_t launch_replay_one(const DbView &db, const uint8_t *d_query, const KParams &kp,
                              const Workspace &ws, int64_t db_index, uint32_t *d_ops, int64_t cap,
                              hs_hit *d_hit, int64_t *d_ops_used, int32_t *d_status, cudaStream_t st);

}  // namespace hs
