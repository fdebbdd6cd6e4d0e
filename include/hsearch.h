/*
 * hsearch.h -- C ABI of the GB300 heuristic protein database search.
 *
 * The method is the randomised sliding-subsequence alignment of Nag &
 * Karforma, "A Space-Efficient Approach towards Distantly Homologous Protein
 * Similarity Searches" (arXiv 1508.06561), in its database-search form:
 * one query is aligned against every database sequence (Sec. III.B.3), each
 * pair with O(1) auxiliary state (Sec. III.B.4), the pairs are ranked by score
 * (Sec. IV) and the best k are returned with their alignments (Fig. 1).
 *
 * Conventions for every entry point:
 *   - Every call returns an int status (HS_OK == 0); nothing is thrown.
 *   - Sequences are residue codes (uint8) in the 24-letter BLOSUM62 order
 *     "ARNDCQEGHILKMFPSTWYVBZX*" (codes 0..23); hs_encode converts ASCII.
 *   - Pointers documented "host" must be host memory; "device" pointers must
 *     be device memory of the current CUDA device.  `stream` is a
 *     cudaStream_t (NULL = the legacy default stream).
 *   - Outputs are caller-allocated; the library keeps no reference to them.
 *   - Results are a pure function of (database, query, params, seed): the
 *     random draws of a pair are keyed by its original database index.
 *   - Hits are ordered by score descending, then database index ascending.
 *   - Scores are int32.  Sequences may be at most HS_MAX_SEQ_LEN long and
 *     penalties at most HS_MAX_PENALTY, which keeps every score in range.
 */
#ifndef HSEARCH_H
#define HSEARCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define HS_OK        0
#define HS_EINVAL    1   /* bad argument (sizes, codes, params, offsets)        */
#define HS_ENOMEM    2   /* device or host allocation failed                    */
#define HS_ECUDA     3   /* a CUDA call failed (no device, launch error, ...)   */
#define HS_ETOOLONG  4   /* a sequence or the query exceeds a supported length  */
#define HS_ETIMEOUT  5   /* a bounded device wait ran out                       */
#define HS_ETRUNC    6   /* an output buffer (ops, workspace) is too small      */
#define HS_EINTERNAL 7   /* replay disagreed with the scan (never expected)     */

#define HS_MAX_SEQ_LEN  1000000
#define HS_MAX_QUERY_LEN 2048
#define HS_MAX_PENALTY  1000
#define HS_MAX_K        4096

#define HS_MODE_DB   0   /* Sec. III.B.3 b: small slides inside large only     */
#define HS_MODE_FULL 1   /* Fig. 1 as printed: small slides across large with
                            any overlap >= 1; pieces may overhang (pair-wise
                            alignment form; not for the batched search)       */

/* alignment run-length ops: op = v & 3, run length = v >> 2 */
#define HS_OP_M 0u       /* query letter against target letter                 */
#define HS_OP_I 1u       /* query letter against a gap in the target           */
#define HS_OP_D 2u       /* target letter against a gap in the query           */

/* ---- parameters (Sec. III.B.1; defaults of Sec. IV) --------------------
 * pgp, gop, gep : periphery, gap-open and gap-extend penalties, >= 0,
 *                 subtracted; an interior gap run of n costs gop+(n-1)*gep.
 * rounds        : AlignSequences' Rounds (>= 1; 1 in database search).
 * lfactor_q16, sfactor_q16, minfactor_q16 : LFactor, SFactor, MinFactor in
 *                 Q16 fixed point (65536 == 1.0), each in [0, 65536].
 * mode          : HS_MODE_DB or HS_MODE_FULL.
 * matrix        : host pointer to a 24x24 row-major int8 table, entry
 *                 [a][b] scoring query letter a against target letter b;
 *                 must be symmetric.  NULL selects the built-in BLOSUM62.  */
typedef struct {
    int32_t pgp, gop, gep, rounds;
    uint32_t lfactor_q16, sfactor_q16, minfactor_q16;
    int32_t mode;
    const int8_t *matrix;
} hs_params;

/* One ranked hit.  The alignment is ops[ops_offset .. ops_offset+ops_len)
 * of the ops buffer and covers both full sequences (its M+I runs sum to the
 * query length, its M+D runs to the target length).  [q_begin, q_end) and
 * [t_begin, t_end) bound the letter-pair columns (all -1 if there are none).*/
typedef struct {
    int64_t db_index;
    int32_t score;
    int32_t q_begin, q_end, t_begin, t_end;
    int32_t ops_len;
    int64_t ops_offset;
} hs_hit;

typedef struct hs_db hs_db;   /* opaque; owns the device copy of a database */

/* The paper's parameter set (Sec. IV): PGP=0, GOP=10, GEP=5, LFactor=0.5,
 * SFactor=1, MinFactor=0.5, Rounds=1 (Sec. III.B.3 a), BLOSUM62. */
void hs_params_default(hs_params *p);

/* ASCII letters -> codes; lower case accepted, any other byte becomes X.
 * ascii and codes_out are host buffers of n bytes. */
int hs_encode(const char *ascii, int64_t n, uint8_t *codes_out);

/* Copies the built-in BLOSUM62 (Henikoff & Henikoff 1992; the matrix of
 * Sec. III.A / III.B.5) into the host buffer out[576]. */
int hs_builtin_matrix(int8_t *out);

/* Checks a parameter block and its matrix without touching the GPU. */
int hs_params_check(const hs_params *p);

/* Database load (the packing step of the search: once per database).
 * codes: host, offsets[n_seqs] residue codes; sequence i is
 * codes[offsets[i] .. offsets[i+1]); offsets: host, n_seqs+1 entries,
 * offsets[0] == 0, non-decreasing; empty sequences are allowed.  The
 * library copies both to the device (the caller keeps its buffers), keeps
 * a longest-first scheduling order of the sequences next to them, and
 * returns a handle in *out.  Errors: HS_EINVAL (bad offsets or codes >= 24),
 * HS_ETOOLONG (a sequence longer than HS_MAX_SEQ_LEN), HS_ENOMEM, HS_ECUDA. */
int hs_db_load(const uint8_t *codes, const int64_t *offsets, int64_t n_seqs,
               void *stream, hs_db **out);

/* A database shard: the same as hs_db_load for sequences whose global
 * database indices start at index_base (>= 0).  Draws, ties and reported
 * hit indices use global indices, so the shards of a database searched
 * separately and merged by (score desc, index asc) give exactly the hits of
 * the whole database (the sharded search of the design notes, Sec. III.B.3
 * applied per shard). */
int hs_db_load_shard(const uint8_t *codes, const int64_t *offsets, int64_t n_seqs, int64_t index_base,
                     void *stream, hs_db **out);

/* Work schedule of the scan (results never depend on it; no counterpart in
 * the paper, whose program visits the database in file order).
 * HS_SCHEDULE_LENGTH (the default after loading): longest targets first,
 * equal lengths in database order, targets of >= 2048 letters one per warp
 * -- the length-binned layout.  The order is built on the device by a
 * stable radix sort of the lengths, with the residues before each schedule
 * position.  HS_SCHEDULE_INPUT: database order, for comparing load balance.
 * Enqueued on `stream` and waited for; allocates scratch for the sort and
 * frees it.  HS_EINVAL, HS_ENOMEM, HS_ECUDA. */
#define HS_SCHEDULE_LENGTH 0
#define HS_SCHEDULE_INPUT  1
int hs_db_set_schedule(hs_db *db, int32_t schedule, void *stream);

/* The current schedule, copied to host buffers (either may be NULL):
 * order_out[n_seqs] = database index at each scan position (shard-local),
 * cumres_out[n_seqs + 1] = residues before each position.  Synchronous. */
int hs_db_get_schedule(const hs_db *db, int32_t *order_out, int64_t *cumres_out);

/* The global index of a database's first sequence (0 unless a shard). */
int hs_db_index_base(const hs_db *db, int64_t *index_base);

/* Number of sequences, residues and the longest length of a database. */
int hs_db_info(const hs_db *db, int64_t *n_seqs, int64_t *n_residues, int32_t *max_len);

/* Releases the handle and its device memory. NULL is ignored. */
void hs_db_free(hs_db *db);

/* Device workspace needed by hs_search_device for a query length and k. */
int hs_search_workspace_size(const hs_db *db, int32_t qlen, int32_t k, size_t *bytes);

/* Ops capacity (entries) that always suffices for k hits of a query length. */
int64_t hs_ops_capacity(int32_t qlen, int32_t k);

/* The search with every buffer on the device (no host copies; asynchronous
 * on `stream`).  Sec. III.B.3: the query d_query[qlen] (device) against every
 * database sequence, then the top min(k, n_seqs) hits with alignments.
 *   d_workspace : device, ws_bytes >= hs_search_workspace_size(...), 256-byte
 *                 aligned; its contents are scratch and are overwritten.
 *   d_hits      : device, min(k, n_seqs) records.
 *   d_ops       : device, ops_cap entries; d_ops_used (device int64) receives
 *                 the entries written.  If ops_cap is too small the status
 *                 word reports HS_ETRUNC.
 *   d_scores    : optional device int32[n_seqs], every pair's score by
 *                 database index (NULL: not written).
 *   d_cells     : optional device int64[n_seqs], the virtual-score cells
 *                 (letter pairs summed) of every pair (NULL: not counted).
 *   d_status    : device int32 receiving HS_OK or the first device-side error.
 *                 A letter code >= 24 in d_query (which the host cannot
 *                 see) is reported here as HS_EINVAL; that column scores 0
 *                 and no memory outside the buffers is read.  HS_ETIMEOUT:
 *                 a wait between the scan's warps ran out (databases with
 *                 many targets of 8,192+ letters share a long pair's steps
 *                 with idle warps at the scan's end; never expected).
 * Host-side argument errors are returned before anything is enqueued. */
int hs_search_device(const hs_db *db, const uint8_t *d_query, int32_t qlen,
                     const hs_params *p, int32_t k, uint64_t seed, void *stream,
                     void *d_workspace, size_t ws_bytes,
                     hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap, int64_t *d_ops_used,
                     int32_t *d_scores, int64_t *d_cells, int32_t *d_status);

/* hs_search_device without allocation (the paper has no counterpart: this
 * serves callers that cannot allocate device memory at search time, such as
 * a process whose memory manager reserved all device memory up front, a
 * serving loop that cannot afford cudaMalloc's implicit synchronisation, or a
 * host that forbids allocation after start-up).  Same arguments and results
 * as hs_search_device, minus the workspace: the scratch is a fixed array of
 * HS_NOALLOC_SCRATCH_BYTES inside the library's device image, which every
 * GPU that loads the library holds until the process exits.  The call makes
 * no cudaMalloc/cudaFree and no allocating library call; the database (from
 * hs_db_load) and every output buffer come from the caller.
 *   - Sizes: HS_ETRUNC if hs_search_workspace_size(db, qlen, k) exceeds
 *     HS_NOALLOC_SCRATCH_BYTES (8 MiB: e.g. ~1.5M targets for a 256-residue
 *     query and k = 100).
 *   - Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before any stream capture.  After a device reset the first
 *     call on the new context looks it up again (the old address is gone).
 *   - Query codes: as for hs_search_device, a code >= 24 in d_query is
 *     reported as HS_EINVAL in *d_status.
 *   - Sharing: all calls on a device use the same array, which keeps the last
 *     call's contents; each call clears what must start at zero.  Calls
 *     whose work overlaps on the GPU (other streams, other threads) race on
 *     it: serialise them. */
#define HS_NOALLOC_SCRATCH_BYTES (8 << 20)
int hs_search_device_noalloc(const hs_db *db, const uint8_t *d_query, int32_t qlen,
                             const hs_params *p, int32_t k, uint64_t seed, void *stream,
                             hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap, int64_t *d_ops_used,
                             int32_t *d_scores, int64_t *d_cells, int32_t *d_status);

/* The same search from host buffers: copies the query (host, qlen codes) in,
 * runs on `stream`, copies the hits and ops back and synchronises.
 *   hits_out : host, room for min(k, n_seqs) records; *n_hits_out receives
 *              the count.
 *   ops_out  : host, ops_cap entries; *ops_used receives the entries needed;
 *              HS_ETRUNC if ops_cap is smaller (hits are still written).
 * Uses a device workspace cached in the handle (grown with cudaMalloc). */
int hs_search(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p,
              int32_t k, uint64_t seed, void *stream,
              hs_hit *hits_out, int32_t *n_hits_out,
              uint32_t *ops_out, int64_t ops_cap, int64_t *ops_used);

/* Batched search: nq queries against the resident database in one
 * persistent scan launch (profiles of all queries, then (query, chunk) work
 * items over the length order, then every query's top k and alignments).
 * Each query's result is exactly hs_search's for that query and its seed.
 * Queries are concatenated: query i is queries[qoffsets[i] .. qoffsets[i+1]).
 * Hits of query i occupy hits[i*k .. i*k + min(k, n_seqs)); their ops
 * offsets index one ops buffer shared by all queries.
 * tuning (optional, NULL = defaults; no counterpart in the paper; every
 * field 0 = its default, results never depend on the tuning):
 *   chunks          chunks per query over the database (<= 8192; default:
 *                   one per ~256 targets, at most 1024);
 *   warps           warps per scan CTA, 24 or 12 (default: the widest that
 *                   fits the class's profile; a value that does not fit is
 *                   ignored);
 *   flat_min_chunks a step is scored as units of the flat list when it has
 *                   at least this many 4-shift chunks (16) ...
 *   flat_max_iters  ... or at most this many iterations per chunk (128);
 *                   the others get a warp's lane grid;
 *   long_len        targets at least this long are taken one per warp (2048).
 * Negative values: HS_EINVAL. */
typedef struct {
    int32_t chunks;
    int32_t warps;
    int32_t flat_min_chunks;
    int32_t flat_max_iters;
    int32_t long_len;
} hs_batch_tuning;

/* Workspace for hs_search_batch_device (total_qlen = sum of query lengths,
 * max_qlen = the longest). */
int hs_search_batch_workspace_size(const hs_db *db, int32_t nq, int64_t total_qlen, int32_t max_qlen,
                                   int32_t k, size_t *bytes);

/* Ops capacity (entries) that always suffices for a batch. */
int64_t hs_batch_ops_capacity(int32_t nq, int64_t total_qlen, int32_t k);

/* Device-resident batched search, asynchronous on `stream` (no host copies,
 * no allocation, so it can be captured in a CUDA graph by the caller).
 *   d_queries, d_qoffsets (int64[nq+1]), d_seeds (uint64[nq]): device; the
 *   offsets must describe queries of 1..max_qlen letters totalling
 *   total_qlen (the host cannot check device data); letter codes >= 24 are
 *   reported as HS_EINVAL in *d_status.
 *   d_hits: nq*k records; d_ops/ops_cap/d_ops_used/d_status as for
 *   hs_search_device. */
int hs_search_batch_device(const hs_db *db, int32_t nq, const uint8_t *d_queries, const int64_t *d_qoffsets,
                           const uint64_t *d_seeds, int64_t total_qlen, int32_t max_qlen,
                           const hs_params *p, int32_t k, const hs_batch_tuning *tuning, void *stream,
                           void *d_workspace, size_t ws_bytes, hs_hit *d_hits, uint32_t *d_ops,
                           int64_t ops_cap, int64_t *d_ops_used, int32_t *d_status);

/* The same from host buffers (queries, qoffsets, seeds, hits_out with room
 * for nq*k records); *n_hits_out = min(k, n_seqs) per query. */
int hs_search_batch(hs_db *db, int32_t nq, const uint8_t *queries, const int64_t *qoffsets,
                    const uint64_t *seeds, const hs_params *p, int32_t k, const hs_batch_tuning *tuning,
                    void *stream, hs_hit *hits_out, int32_t *n_hits_out, uint32_t *ops_out,
                    int64_t ops_cap, int64_t *ops_used);

/* Threshold reporting (Sec. IV reports the hits above a chosen threshold
 * score).  The same search as hs_search, keeping every pair that scores
 * >= threshold, ranked, at most max_hits (<= HS_MAX_K) of them with their
 * alignments.  *n_above_out receives the number of pairs at or above the
 * threshold (more than *n_hits_out when max_hits truncated the list). */
int hs_search_threshold(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p,
                        int32_t threshold, int32_t max_hits, uint64_t seed, void *stream,
                        hs_hit *hits_out, int32_t *n_hits_out, int64_t *n_above_out,
                        uint32_t *ops_out, int64_t ops_cap, int64_t *ops_used);

/* One pair replayed alone (Fig. 1's AlignSequences for the query and
 * database sequence db_index, with the same draws as hs_search): its score
 * and its alignment ops (host buffer of `cap` entries).  db_index is the
 * global index (as reported in hits; shards subtract their index base). */
int hs_get_alignment(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p,
                     uint64_t seed, int64_t db_index, void *stream,
                     uint32_t *ops_out, int64_t cap, int32_t *score_out,
                     int64_t *ops_len_out, hs_hit *hit_out);

/* Bytes hs_search moves per call: host->device (the query) and
 * device->host (hits, status and the ops region), for a query length and k. */
int hs_search_transfer_bytes(int32_t qlen, int32_t k, int64_t *h2d, int64_t *d2h);

/* Tracing hook (no counterpart in the paper; for profiling).  When set on a
 * database, every later search on it records scan_start / scan_stop (two
 * cudaEvent_t created by the caller, or NULL) on its stream around the
 * database scan, and stores in `launches` the number of kernels the search
 * launched.  With pack_shifts nonzero, a database-mode hs_search_device that
 * counts cells (d_cells) stores per pair cells + (shifts << 40) instead,
 * shifts being the number of shifts whose virtual score was taken
 * (sum over steps of ls - ss + 1; cells stay below 2^40).  Zero-initialise
 * the struct.  It must stay valid while set; NULL clears the hook. */
typedef struct {
    void *scan_start, *scan_stop;
    int32_t launches;
    int32_t pack_shifts;
} hs_trace;
int hs_db_set_trace(hs_db *db, hs_trace *trace);

/* Static message for a status code. */
const char *hs_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* HSEARCH_H */
