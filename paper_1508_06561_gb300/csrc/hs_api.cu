// hs_api.cu -- host runtime behind the C ABI of include/hsearch.h.
// Database load (packing + length order), parameter checks, workspace
// carve-up and the search pipeline: profile -> scan -> top-k -> replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hs_internal.h"

namespace hs {

// BLOSUM62 (Henikoff & Henikoff, PNAS 1992), rows and columns in the order
// A R N D C Q E G H I L K M F P S T W Y V B Z X *.
static const int8_t kBlosum62[kNSym * kNSym] = {
    4, -1, -2, -2, 0, -1, -1, 0, -2, -1, -1, -1, -1, -2, -1, 1, 0, -3, -2, 0, -2, -1, 0, -4,
    -1, 5, 0, -2, -3, 1, 0, -2, 0, -3, -2, 2, -1, -3, -2, -1, -1, -3, -2, -3, -1, 0, -1, -4,
    -2, 0, 6, 1, -3, 0, 0, 0, 1, -3, -3, 0, -2, -3, -2, 1, 0, -4, -2, -3, 3, 0, -1, -4,
    -2, -2, 1, 6, -3, 0, 2, -1, -1, -3, -4, -1, -3, -3, -1, 0, -1, -4, -3, -3, 4, 1, -1, -4,
    0, -3, -3, -3, 9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1, -3, -3, -2, -4,
    -1, 1, 0, 0, -3, 5, 2, -2, 0, -3, -2, 1, 0, -3, -1, 0, -1, -2, -1, -2, 0, 3, -1, -4,
    -1, 0, 0, 2, -4, 2, 5, -2, 0, -3, -3, 1, -2, -3, -1, 0, -1, -3, -2, -2, 1, 4, -1, -4,
    0, -2, 0, -1, -3, -2, -2, 6, -2, -4, -4, -2, -3, -3, -2, 0, -2, -2, -3, -3, -1, -2, -1, -4,
    -2, 0, 1, -1, -3, 0, 0, -2, 8, -3, -3, -1, -2, -1, -2, -1, -2, -2, 2, -3, 0, 0, -1, -4,
    -1, -3, -3, -3, -1, -3, -3, -4, -3, 4, 2, -3, 1, 0, -3, -2, -1, -3, -1, 3, -3, -3, -1, -4,
    -1, -2, -3, -4, -1, -2, -3, -4, -3, 2, 4, -2, 2, 0, -3, -2, -1, -2, -1, 1, -4, -3, -1, -4,
    -1, 2, 0, -1, -3, 1, 1, -2, -1, -3, -2, 5, -1, -3, -1, 0, -1, -3, -2, -2, 0, 1, -1, -4,
    -1, -1, -2, -3, -1, 0, -2, -3, -2, 1, 2, -1, 5, 0, -2, -1, -1, -1, -1, 1, -3, -1, -1, -4,
    -2, -3, -3, -3, -2, -3, -3, -3, -1, 0, 0, -3, 0, 6, -4, -2, -2, 1, 3, -1, -3, -3, -1, -4,
    -1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4, 7, -1, -1, -4, -3, -2, -2, -1, -2, -4,
    1, -1, 1, 0, -1, 0, 0, 0, -1, -2, -2, 0, -1, -2, -1, 4, 1, -3, -2, -2, 0, 0, 0, -4,
    0, -1, 0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1, 1, 5, -2, -2, 0, -1, -1, 0, -4,
    -3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1, 1, -4, -3, -2, 11, 2, -3, -4, -3, -2, -4,
    -2, -2, -2, -3, -2, -1, -2, -3, 2, -1, -1, -2, -1, 3, -3, -2, -2, 2, 7, -1, -3, -2, -1, -4,
    0, -3, -3, -3, -1, -2, -2, -3, -3, 3, 1, -2, 1, -1, -2, -2, 0, -3, -1, 4, -3, -2, -1, -4,
    -2, -1, 3, 4, -3, 0, 1, -1, 0, -3, -4, 0, -3, -3, -2, 0, -1, -4, -3, -3, 4, 1, -1, -4,
    -1, 0, 0, 1, -3, 3, 4, -2, 0, -3, -3, 1, -1, -3, -1, 0, -1, -3, -2, -2, 1, 4, -1, -4,
    0, -1, -1, -1, -2, -1, -1, -1, -1, -1, -1, -1, -1, -1, -2, 0, 0, -2, -1, -1, -1, -1, -1, -4,
    -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, 1,
};

static const char kLetters[kNSym + 1] = "ARNDCQEGHILKMFPSTWYVBZX*";

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// NVTX ranges around the host side of each phase (load, search, and the
// enqueue of profile+scan, top-k and replay), for timeline profilers; free
// when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

int64_t slot_stride_for(int32_t qlen) { return 2LL * qlen + 4; }

size_t workspace_bytes(int64_t n, int32_t qlen, int32_t k)
{
    size_t b = 0;
    b += align256(sizeof(uint32_t) * 2 * (size_t)profile_words(qlen));
    b += align256(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1));
    b += align256(sizeof(uint32_t) * kNumCounters);
    b += align256(sizeof(uint64_t) * (size_t)kTopkCtas * std::max(k, 1));
    b += align256(sizeof(int64_t) * (size_t)std::max(k, 1));
    b += align256(sizeof(int32_t) * (size_t)std::max(k, 1));
    b += align256(sizeof(uint32_t) * (size_t)std::max(k, 1) * (size_t)slot_stride_for(qlen));
    b += align256(sizeof(int32_t) * (size_t)std::max(k, 1));
    return b;
}

Workspace carve_workspace(void *base, int64_t n, int32_t qlen, int32_t k)
{
    Workspace w;
    char *p = static_cast<char *>(base);
    auto take = [&](size_t bytes) { char *r = p; p += align256(bytes); return r; };
    w.prof = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * 2 * (size_t)profile_words(qlen)));
    w.scores = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
    w.counters = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * kNumCounters));
    w.cand = reinterpret_cast<uint64_t *>(take(sizeof(uint64_t) * (size_t)kTopkCtas * std::max(k, 1)));
    w.hit_idx = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (size_t)std::max(k, 1)));
    w.hit_score = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)std::max(k, 1)));
    w.slot_stride = slot_stride_for(qlen);
    w.slots = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)std::max(k, 1) * (size_t)w.slot_stride));
    w.slot_len = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * (size_t)std::max(k, 1)));
    w.topk_ctas = kTopkCtas;
    w.k = k;
    return w;
}

// Fault injection for tests: while HS_FAIL_ALLOC is set (non-empty) in the
// environment, every allocation the library makes fails as if memory were
// exhausted, so the HS_ENOMEM paths can be exercised without exhausting a
// GPU.  They release what they took and leave handles usable.
static bool alloc_refused()
{
    const char *v = std::getenv("HS_FAIL_ALLOC");
    return v && *v;
}

template <class T> static cudaError_t dev_malloc(T **p, size_t bytes)
{
    if (alloc_refused()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

template <class T> static cudaError_t host_malloc(T **p, size_t bytes)
{
    if (alloc_refused()) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, bytes);
}

static int from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return HS_OK;
    if (e == cudaErrorMemoryAllocation) return HS_ENOMEM;
    return HS_ECUDA;
}

static int make_kparams(const hs_params *p, int32_t qlen, uint64_t seed, KParams *kp)
{
    int rc = hs_params_check(p);
    if (rc != HS_OK) return rc;
    const int8_t *m = p->matrix ? p->matrix : kBlosum62;
    int lo = 127, hi = -128;
    for (int i = 0; i < kNSym * kNSym; i++) {
        kp->m[i] = m[i];
        lo = std::min<int>(lo, m[i]);
        hi = std::max<int>(hi, m[i]);
    }
    SParams &sp = kp->s;
    sp.bias = -lo;
    const int range = hi - lo;
    sp.flush = range == 0 ? 255 : std::max(1, 255 / range);
    sp.pgp = p->pgp; sp.gop = p->gop; sp.gep = p->gep; sp.rounds = p->rounds;
    sp.lf_q16 = p->lfactor_q16; sp.sf_q16 = p->sfactor_q16; sp.minf_q16 = p->minfactor_q16;
    sp.qlen = qlen;
    sp.seed = seed;
    sp.index_base = 0;
    sp.min_score = INT_MIN;
    sp.mode = p->mode;
    sp.pair16 = (int64_t)range * (qlen + 3) <= 65535;
    sp.pack_shifts = 0;
    sp.flat_min_chunks = kFlatMinChunks;
    sp.flat_max_iters = kFlatMaxIters;
    sp.help_min_units = kHelpMinUnits;
    return HS_OK;
}

}  // namespace hs

using namespace hs;

struct hs_db {
    int64_t n = 0, nres = 0;
    int64_t index_base = 0;                 // global index of sequence 0 (database shards)
    int32_t maxlen = 0;
    int device = 0, num_sms = 0;
    uint8_t *d_codes = nullptr;
    int64_t *d_offsets = nullptr;
    int32_t *d_order = nullptr;
    int64_t *d_cumres = nullptr;            // residues before each position of the schedule
    std::vector<int32_t> sorted_len;        // lengths in schedule order (non-increasing unless input order)
    int32_t schedule = HS_SCHEDULE_LENGTH;
    // host-API state (grown on demand)
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    char *d_io = nullptr;                   // query | hits | meta | ops
    size_t io_bytes = 0;
    char *h_io = nullptr;                   // pinned mirror of d_io
    size_t h_io_bytes = 0;
    hs_trace *trace = nullptr;              // optional tracing hook
};

extern "C" {

void hs_params_default(hs_params *p)
{
    if (!p) return;
    p->pgp = 0; p->gop = 10; p->gep = 5; p->rounds = 1;
    p->lfactor_q16 = 32768; p->sfactor_q16 = 65536; p->minfactor_q16 = 32768;
    p->mode = HS_MODE_DB;
    p->matrix = nullptr;
}

int hs_encode(const char *ascii, int64_t n, uint8_t *codes_out)
{
    if (n < 0 || (n > 0 && (!ascii || !codes_out))) return HS_EINVAL;
    uint8_t table[256];
    for (int c = 0; c < 256; c++) table[c] = 22;   // X
    for (int i = 0; i < kNSym; i++) {
        table[(unsigned char)kLetters[i]] = (uint8_t)i;
        if (kLetters[i] >= 'A' && kLetters[i] <= 'Z') table[(unsigned char)(kLetters[i] - 'A' + 'a')] = (uint8_t)i;
    }
    for (int64_t i = 0; i < n; i++) codes_out[i] = table[(unsigned char)ascii[i]];
    return HS_OK;
}

int hs_builtin_matrix(int8_t *out)
{
    if (!out) return HS_EINVAL;
    std::memcpy(out, kBlosum62, sizeof(kBlosum62));
    return HS_OK;
}

int hs_params_check(const hs_params *p)
{
    if (!p) return HS_EINVAL;
    if (p->pgp < 0 || p->gop < 0 || p->gep < 0) return HS_EINVAL;
    if (p->pgp > HS_MAX_PENALTY || p->gop > HS_MAX_PENALTY || p->gep > HS_MAX_PENALTY) return HS_EINVAL;
    if (p->rounds < 1 || p->rounds > 1000) return HS_EINVAL;
    if (p->lfactor_q16 > 65536 || p->sfactor_q16 > 65536 || p->minfactor_q16 > 65536) return HS_EINVAL;
    if (p->mode != HS_MODE_DB && p->mode != HS_MODE_FULL) return HS_EINVAL;
    if (p->matrix) {
        for (int a = 0; a < kNSym; a++)
            for (int b = 0; b < a; b++)
                if (p->matrix[a * kNSym + b] != p->matrix[b * kNSym + a]) return HS_EINVAL;
    }
    return HS_OK;
}

const char *hs_strerror(int status)
{
    switch (status) {
    case HS_OK: return "ok";
    case HS_EINVAL: return "invalid argument";
    case HS_ENOMEM: return "out of memory";
    case HS_ECUDA: return "CUDA error";
    case HS_ETOOLONG: return "sequence or query too long";
    case HS_ETIMEOUT: return "device wait timed out";
    case HS_ETRUNC: return "output buffer too small";
    case HS_EINTERNAL: return "internal error: replay disagrees with scan";
    default: return "unknown status";
    }
}

void hs_db_free(hs_db *db)
{
    if (!db) return;
    cudaFree(db->d_codes);
    cudaFree(db->d_offsets);
    cudaFree(db->d_order);
    cudaFree(db->d_cumres);
    cudaFree(db->d_ws);
    cudaFree(db->d_io);
    if (db->h_io) cudaFreeHost(db->h_io);
    delete db;
}

int hs_db_load(const uint8_t *codes, const int64_t *offsets, int64_t n_seqs, void *stream, hs_db **out)
{
    return hs_db_load_shard(codes, offsets, n_seqs, 0, stream, out);
}

int hs_db_load_shard(const uint8_t *codes, const int64_t *offsets, int64_t n_seqs, int64_t index_base,
                     void *stream, hs_db **out)
{
    NvtxRange r("hs_db_load");
    if (index_base < 0 || index_base > (int64_t)INT32_MAX) return HS_EINVAL;
    if (!out || !offsets || n_seqs < 0 || n_seqs > INT32_MAX - 1) return HS_EINVAL;
    *out = nullptr;
    if (offsets[0] != 0) return HS_EINVAL;
    int32_t maxlen = 0;
    for (int64_t i = 0; i < n_seqs; i++) {
        const int64_t len = offsets[i + 1] - offsets[i];
        if (len < 0) return HS_EINVAL;
        if (len > HS_MAX_SEQ_LEN) return HS_ETOOLONG;
        maxlen = std::max<int32_t>(maxlen, (int32_t)len);
    }
    const int64_t nres = offsets[n_seqs];
    if (nres > 0 && !codes) return HS_EINVAL;
    for (int64_t i = 0; i < nres; i++)
        if (codes[i] >= kNSym) return HS_EINVAL;

    hs_db *db = alloc_refused() ? nullptr : new (std::nothrow) hs_db();
    if (!db) return HS_ENOMEM;
    db->n = n_seqs;
    db->nres = nres;
    db->maxlen = maxlen;
    db->index_base = index_base;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&db->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&db->num_sms, cudaDevAttrMultiProcessorCount, db->device);
    if (e != cudaSuccess) { hs_db_free(db); return from_cuda(e); }

    e = dev_malloc(&db->d_codes, (size_t)nres + kCodesPad);
    if (e == cudaSuccess) e = dev_malloc(&db->d_offsets, sizeof(int64_t) * (size_t)(n_seqs + 1));
    if (e == cudaSuccess) e = dev_malloc(&db->d_order, sizeof(int32_t) * (size_t)std::max<int64_t>(n_seqs, 1));
    if (e == cudaSuccess) e = dev_malloc(&db->d_cumres, sizeof(int64_t) * (size_t)(n_seqs + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(db->d_codes + nres, 0, kCodesPad, st);
    if (e == cudaSuccess && nres > 0) e = cudaMemcpyAsync(db->d_codes, codes, (size_t)nres, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db->d_offsets, offsets, sizeof(int64_t) * (size_t)(n_seqs + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { hs_db_free(db); return from_cuda(e); }
    const int rc = hs_db_set_schedule(db, HS_SCHEDULE_LENGTH, stream);
    if (rc != HS_OK) { hs_db_free(db); return rc; }
    *out = db;
    return HS_OK;
}

int hs_db_set_schedule(hs_db *db, int32_t schedule, void *stream)
{
    NvtxRange r("hs_db_set_schedule");
    if (!db || (schedule != HS_SCHEDULE_LENGTH && schedule != HS_SCHEDULE_INPUT)) return HS_EINVAL;
    const int64_t n = db->n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the order is built on the device (hs_sort.cu); the host keeps the
    // lengths in schedule order for the role split and the long prefix
    void *scratch = nullptr;
    int32_t *d_len = nullptr;
    std::vector<int32_t> len((size_t)n);
    cudaError_t e = dev_malloc(&scratch, schedule_scratch_bytes(n));
    if (e == cudaSuccess) e = dev_malloc(&d_len, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1));
    if (e == cudaSuccess)
        e = build_schedule(db->d_offsets, n, db->maxlen, schedule == HS_SCHEDULE_LENGTH, db->d_order, db->d_cumres,
                           d_len, scratch, st);
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(len.data(), d_len, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(scratch);
    cudaFree(d_len);
    if (e != cudaSuccess) return from_cuda(e);
    db->sorted_len.swap(len);
    db->schedule = schedule;
    return HS_OK;
}

int hs_db_get_schedule(const hs_db *db, int32_t *order_out, int64_t *cumres_out)
{
    if (!db) return HS_EINVAL;
    cudaError_t e = cudaSuccess;
    if (order_out && db->n > 0)
        e = cudaMemcpy(order_out, db->d_order, sizeof(int32_t) * (size_t)db->n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && cumres_out)
        e = cudaMemcpy(cumres_out, db->d_cumres, sizeof(int64_t) * (size_t)(db->n + 1), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HS_OK : from_cuda(e);
}

int hs_db_index_base(const hs_db *db, int64_t *index_base)
{
    if (!db || !index_base) return HS_EINVAL;
    *index_base = db->index_base;
    return HS_OK;
}

int hs_db_info(const hs_db *db, int64_t *n_seqs, int64_t *n_residues, int32_t *max_len)
{
    if (!db) return HS_EINVAL;
    if (n_seqs) *n_seqs = db->n;
    if (n_residues) *n_residues = db->nres;
    if (max_len) *max_len = db->maxlen;
    return HS_OK;
}

int hs_search_workspace_size(const hs_db *db, int32_t qlen, int32_t k, size_t *bytes)
{
    if (!db || !bytes || qlen < 1 || k < 0) return HS_EINVAL;
    if (qlen > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
    if (k > HS_MAX_K) return HS_EINVAL;
    *bytes = workspace_bytes(db->n, qlen, k);
    return HS_OK;
}

int64_t hs_ops_capacity(int32_t qlen, int32_t k)
{
    if (qlen < 1 || k < 0) return 0;
    return (int64_t)k * slot_stride_for(qlen);
}

// The search pipeline on the device: profile -> scan -> top-k -> replay,
// plus (threshold search) the count of pairs scoring >= min_score.
static int run_search(const hs_db *db, const uint8_t *d_query, int32_t qlen, const hs_params *p, int32_t k,
                      uint64_t seed, int32_t min_score, void *stream, void *d_workspace, size_t ws_bytes,
                      hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap, int64_t *d_ops_used, int32_t *d_scores,
                      int64_t *d_cells, int32_t *d_status, int64_t *d_count)
{
    if (!db || !d_query || !p || !d_workspace || !d_status) return HS_EINVAL;
    if (qlen < 1) return HS_EINVAL;
    if (qlen > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
    if (k < 0 || k > HS_MAX_K || ops_cap < 0) return HS_EINVAL;
    const int32_t nhits = (int32_t)std::min<int64_t>(k, db->n);
    if (nhits > 0 && (!d_hits || !d_ops_used || (ops_cap > 0 && !d_ops))) return HS_EINVAL;
    if (((uintptr_t)d_workspace & 255) != 0) return HS_EINVAL;
    if (ws_bytes < workspace_bytes(db->n, qlen, k)) return HS_ETRUNC;
    KParams kp;
    int rc = make_kparams(p, qlen, seed, &kp);
    if (rc != HS_OK) return rc;
    kp.s.index_base = db->index_base;
    kp.s.min_score = min_score;
    kp.s.pack_shifts = db->trace && db->trace->pack_shifts && d_cells && kp.s.mode == HS_MODE_DB;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Workspace ws = carve_workspace(d_workspace, db->n, qlen, k);
    if (d_scores) ws.scores = d_scores;
    cudaError_t e = cudaMemsetAsync(ws.counters, 0, sizeof(uint32_t) * kNumCounters, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return from_cuda(e);
    if (nhits == 0 && d_ops_used) {
        e = cudaMemsetAsync(d_ops_used, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (d_count) {
        e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (db->n == 0) return HS_OK;

    // role split and the long prefix in the length order (unused in input order)
    const auto &L = db->sorted_len;
    const bool input_order = db->schedule == HS_SCHEDULE_INPUT;
    const int64_t split = input_order ? 0 :
        std::partition_point(L.begin(), L.end(), [&](int32_t x) { return x >= qlen; }) - L.begin();
    const int64_t long_end = input_order ? 0 :
        std::partition_point(L.begin(), L.end(), [&](int32_t x) { return x >= kLongLen; }) - L.begin();
    // At least one target of kHelpLen letters per SM: some pair's chain of
    // steps may outlast the rest of the scan, so idle warps help it (the
    // plain swissprot-like database has 44 such targets, the bimodal one 8,999).
    const bool share_steps = !input_order &&
        std::partition_point(L.begin(), L.end(), [&](int32_t x) { return x >= kHelpLen; }) - L.begin() >= db->num_sms;
    DbView v{db->d_codes, db->d_offsets, db->d_order, db->n};
    ScanTrace tr{nullptr, nullptr};
    if (db->trace) {
        tr.start = static_cast<cudaEvent_t>(db->trace->scan_start);
        tr.stop = static_cast<cudaEvent_t>(db->trace->scan_stop);
    }
    int launches = 0;
    {
        NvtxRange r("hs.scan");
        e = launch_scan(v, split, long_end, d_query, kp, ws, d_cells, d_status, db->num_sms, st,
                        db->trace ? &tr : nullptr, &launches, input_order, share_steps);
        if (e == cudaSuccess && d_count)
            e = launch_count_at_least(ws.scores, db->n, min_score, d_count, db->num_sms, st, &launches);
    }
    if (e == cudaSuccess && nhits > 0) {
        NvtxRange r("hs.topk");
        e = launch_topk(ws, db->n, nhits, st, &launches);
    }
    if (e == cudaSuccess && nhits > 0) {
        NvtxRange r("hs.replay");
        e = launch_replay(v, d_query, kp, ws, nhits, d_hits, d_ops, ops_cap, d_ops_used, d_status, st,
                          &launches);
    }
    if (db->trace) db->trace->launches = launches;
    return from_cuda(e);
}

int hs_search_device(const hs_db *db, const uint8_t *d_query, int32_t qlen, const hs_params *p, int32_t k,
                     uint64_t seed, void *stream, void *d_workspace, size_t ws_bytes, hs_hit *d_hits,
                     uint32_t *d_ops, int64_t ops_cap, int64_t *d_ops_used, int32_t *d_scores,
                     int64_t *d_cells, int32_t *d_status)
{
    NvtxRange r("hs_search_device");
    return run_search(db, d_query, qlen, p, k, seed, INT_MIN, stream, d_workspace, ws_bytes, d_hits, d_ops,
                      ops_cap, d_ops_used, d_scores, d_cells, d_status, nullptr);
}

// host-API buffers: [query | hits | ops_used, status | ops]
struct IoLayout {
    size_t q, hits, meta, ops, total;
};
static IoLayout io_layout(int32_t qlen, int32_t k)
{
    IoLayout l;
    l.q = 0;
    l.hits = align256((size_t)qlen);
    l.meta = l.hits + align256(sizeof(hs_hit) * (size_t)std::max(k, 1));
    l.ops = l.meta + 256;
    l.total = l.ops + align256(sizeof(uint32_t) * (size_t)std::max<int64_t>(hs_ops_capacity(qlen, k), 1));
    return l;
}

static int ensure_host_state(hs_db *db, size_t ws_need, size_t io_need)
{
    cudaError_t e = cudaSuccess;
    if (db->ws_bytes < ws_need) {
        cudaFree(db->d_ws);
        db->d_ws = nullptr;
        db->ws_bytes = 0;
        e = dev_malloc(&db->d_ws, ws_need);
        if (e != cudaSuccess) return from_cuda(e);
        db->ws_bytes = ws_need;
    }
    if (db->io_bytes < io_need) {
        cudaFree(db->d_io);
        db->d_io = nullptr;
        db->io_bytes = 0;
        e = dev_malloc(&db->d_io, io_need);
        if (e != cudaSuccess) return from_cuda(e);
        db->io_bytes = io_need;
    }
    if (db->h_io_bytes < io_need) {
        if (db->h_io) cudaFreeHost(db->h_io);
        db->h_io = nullptr;
        db->h_io_bytes = 0;
        e = host_malloc(&db->h_io, io_need);
        if (e != cudaSuccess) return from_cuda(e);
        db->h_io_bytes = io_need;
    }
    return HS_OK;
}

int hs_search_transfer_bytes(int32_t qlen, int32_t k, int64_t *h2d, int64_t *d2h)
{
    if (qlen < 1 || k < 0 || !h2d || !d2h) return HS_EINVAL;
    const IoLayout l = io_layout(qlen, k);
    *h2d = qlen;
    *d2h = (int64_t)(l.total - l.hits);
    return HS_OK;
}

int hs_db_set_trace(hs_db *db, hs_trace *trace)
{
    if (!db) return HS_EINVAL;
    db->trace = trace;
    return HS_OK;
}

// Host-buffer search (query in, hits and ops out, synchronised); with a
// threshold, only hits scoring >= min_score are kept and *n_above receives
// the number of pairs at or above it.
static int run_host_search(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p, int32_t k,
                           uint64_t seed, int32_t min_score, bool threshold, void *stream, hs_hit *hits_out,
                           int32_t *n_hits_out, uint32_t *ops_out, int64_t ops_cap, int64_t *ops_used,
                           int64_t *n_above)
{
    NvtxRange r(threshold ? "hs_search_threshold" : "hs_search");
    if (!db || !query || !p || !n_hits_out || !ops_used) return HS_EINVAL;
    if (qlen < 1) return HS_EINVAL;
    if (qlen > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
    if (k < 0 || k > HS_MAX_K || ops_cap < 0) return HS_EINVAL;
    const int32_t nhits = (int32_t)std::min<int64_t>(k, db->n);
    if (nhits > 0 && !hits_out) return HS_EINVAL;
    for (int32_t i = 0; i < qlen; i++)
        if (query[i] >= kNSym) return HS_EINVAL;
    int rc = hs_params_check(p);
    if (rc != HS_OK) return rc;
    const IoLayout l = io_layout(qlen, k);
    rc = ensure_host_state(db, workspace_bytes(db->n, qlen, k), l.total);
    if (rc != HS_OK) return rc;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *h = db->h_io, *d = db->d_io;
    std::memcpy(h + l.q, query, (size_t)qlen);
    cudaError_t e = cudaMemcpyAsync(d + l.q, h + l.q, (size_t)qlen, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    const int64_t cap = hs_ops_capacity(qlen, k);
    rc = run_search(db, reinterpret_cast<const uint8_t *>(d + l.q), qlen, p, k, seed, min_score, stream, db->d_ws,
                    db->ws_bytes, reinterpret_cast<hs_hit *>(d + l.hits), reinterpret_cast<uint32_t *>(d + l.ops),
                    cap, reinterpret_cast<int64_t *>(d + l.meta), nullptr, nullptr,
                    reinterpret_cast<int32_t *>(d + l.meta + 8),
                    threshold ? reinterpret_cast<int64_t *>(d + l.meta + 16) : nullptr);
    if (rc != HS_OK) return rc;
    // one copy back: hits, ops_used/status/count and the packed ops
    e = cudaMemcpyAsync(h + l.hits, d + l.hits, l.total - l.hits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    int64_t used, count = 0;
    int32_t status;
    std::memcpy(&used, h + l.meta, sizeof(used));
    std::memcpy(&status, h + l.meta + 8, sizeof(status));
    if (threshold) std::memcpy(&count, h + l.meta + 16, sizeof(count));
    if (nhits == 0) used = 0;
    if (status != HS_OK) return status;
    const hs_hit *dh = reinterpret_cast<const hs_hit *>(h + l.hits);
    int32_t keep = nhits;
    if (threshold) {                        // hits are ranked: keep the prefix above the threshold
        keep = 0;
        while (keep < nhits && dh[keep].score >= min_score) keep++;
        *n_above = count;
    }
    if (keep > 0) std::memcpy(hits_out, dh, sizeof(hs_hit) * (size_t)keep);
    *n_hits_out = keep;
    *ops_used = used;
    if (used > ops_cap) return HS_ETRUNC;
    if (used > 0) std::memcpy(ops_out, h + l.ops, sizeof(uint32_t) * (size_t)used);
    return HS_OK;
}

int hs_search(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p, int32_t k, uint64_t seed,
              void *stream, hs_hit *hits_out, int32_t *n_hits_out, uint32_t *ops_out, int64_t ops_cap,
              int64_t *ops_used)
{
    return run_host_search(db, query, qlen, p, k, seed, INT_MIN, false, stream, hits_out, n_hits_out, ops_out,
                           ops_cap, ops_used, nullptr);
}

int hs_search_threshold(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p, int32_t threshold,
                        int32_t max_hits, uint64_t seed, void *stream, hs_hit *hits_out, int32_t *n_hits_out,
                        int64_t *n_above_out, uint32_t *ops_out, int64_t ops_cap, int64_t *ops_used)
{
    if (!n_above_out) return HS_EINVAL;
    return run_host_search(db, query, qlen, p, max_hits, seed, threshold, true, stream, hits_out, n_hits_out,
                           ops_out, ops_cap, ops_used, n_above_out);
}

// ---------------------------------------------------------------------------
// Batched search: many queries, one persistent scan launch.
// ---------------------------------------------------------------------------
static size_t batch_layout(int64_t n, int32_t nq, int64_t total_qlen, int32_t max_qlen, int32_t k, char *base,
                           BatchLayout *bl)
{
    char *p = base;
    size_t used = 0;
    auto take = [&](size_t bytes) {
        char *r = p ? p + used : nullptr;
        used += align256(bytes);
        return r;
    };
    const size_t kk = (size_t)std::max(k, 1), qq = (size_t)std::max(nq, 1);
    BatchLayout b = {};
    b.counter_bytes = (int64_t)(sizeof(unsigned) * (5 + qq));
    b.counters = reinterpret_cast<unsigned *>(take((size_t)b.counter_bytes));
    b.qlist = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * 2 * qq));
    b.prof_off = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * qq));
    b.prof = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * 2 * kNSym * (size_t)(total_qlen + 17 * qq)));
    b.bounds = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (kMaxChunks + 1)));
    b.scores = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * qq * (size_t)std::max<int64_t>(n, 1)));
    b.cand = reinterpret_cast<uint64_t *>(take(sizeof(uint64_t) * qq * kTopkCtas * kk));
    b.hit_idx = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * qq * kk));
    b.hit_score = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * qq * kk));
    b.slot_stride = slot_stride_for(std::max(max_qlen, 1));
    b.slots = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * qq * kk * (size_t)b.slot_stride));
    b.slot_len = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * qq * kk));
    if (b.counters) {
        b.item_ctrs = b.counters;
        b.class_counts = b.counters + 2;
        b.replay_ticket = b.counters + 4;
        b.topk_tickets = b.counters + 5;
    }
    b.nq = nq;
    b.max_qlen = max_qlen;
    if (bl) *bl = b;
    return used;
}

int hs_search_batch_workspace_size(const hs_db *db, int32_t nq, int64_t total_qlen, int32_t max_qlen, int32_t k,
                                   size_t *bytes)
{
    if (!db || !bytes || nq < 0 || total_qlen < 0 || max_qlen < 1 || k < 0 || k > HS_MAX_K) return HS_EINVAL;
    if (max_qlen > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
    *bytes = batch_layout(db->n, nq, total_qlen, max_qlen, k, nullptr, nullptr);
    return HS_OK;
}

int64_t hs_batch_ops_capacity(int32_t nq, int64_t total_qlen, int32_t k)
{
    if (nq < 0 || total_qlen < 0 || k < 0) return 0;
    return (int64_t)k * (2 * total_qlen + 4LL * nq);
}

int hs_search_batch_device(const hs_db *db, int32_t nq, const uint8_t *d_queries, const int64_t *d_qoffsets,
                           const uint64_t *d_seeds, int64_t total_qlen, int32_t max_qlen, const hs_params *p,
                           int32_t k, const hs_batch_tuning *tuning, void *stream, void *d_workspace,
                           size_t ws_bytes, hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap,
                           int64_t *d_ops_used, int32_t *d_status)
{
    NvtxRange r("hs_search_batch_device");
    if (!db || !p || !d_workspace || !d_status || nq < 0) return HS_EINVAL;
    if (nq > 0 && (!d_queries || !d_qoffsets || !d_seeds)) return HS_EINVAL;
    if (max_qlen < 1 || total_qlen < nq) return HS_EINVAL;
    if (max_qlen > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
    if (k < 0 || k > HS_MAX_K || ops_cap < 0) return HS_EINVAL;
    // default: about 256 targets per chunk, at most kDefaultChunks (the
    // 570k-target database's best); a small database gets a few large
    // chunks, so that an item is not a handful of pairs behind a profile copy
    // and a CTA barrier
    const int32_t nchunk = tuning && tuning->chunks > 0
                               ? tuning->chunks
                               : (int32_t)std::max<int64_t>(1, std::min<int64_t>(kDefaultChunks, (db->n + 255) / 256));
    if (nchunk > kMaxChunks) return HS_EINVAL;
    if (tuning && (tuning->warps < 0 || tuning->flat_min_chunks < 0 || tuning->flat_max_iters < 0 ||
                   tuning->long_len < 0))
        return HS_EINVAL;
    const int warps = tuning ? tuning->warps : 0;
    const int32_t long_len = tuning && tuning->long_len > 0 ? tuning->long_len : kLongLen;
    const int32_t nhits = (int32_t)std::min<int64_t>(k, db->n);
    if (nhits > 0 && nq > 0 && (!d_hits || !d_ops_used || (ops_cap > 0 && !d_ops))) return HS_EINVAL;
    if (((uintptr_t)d_workspace & 255) != 0) return HS_EINVAL;
    BatchLayout bl;
    const size_t need = batch_layout(db->n, nq, total_qlen, max_qlen, k, static_cast<char *>(d_workspace), &bl);
    if (ws_bytes < need) return HS_ETRUNC;
    KParams kp;
    int rc = make_kparams(p, max_qlen, 0, &kp);
    if (rc != HS_OK) return rc;
    if (p->mode != HS_MODE_DB) return HS_EINVAL;    // the batched scan is the database-search form
    kp.s.index_base = db->index_base;
    if (tuning && tuning->flat_min_chunks > 0) kp.s.flat_min_chunks = tuning->flat_min_chunks;
    if (tuning && tuning->flat_max_iters > 0) kp.s.flat_max_iters = tuning->flat_max_iters;
    bl.queries = d_queries;
    bl.qoffsets = d_qoffsets;
    bl.seeds = d_seeds;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(bl.counters, 0, (size_t)bl.counter_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess && d_ops_used) e = cudaMemsetAsync(d_ops_used, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return from_cuda(e);
    if (db->n == 0 || nq == 0) return HS_OK;

    const auto &L = db->sorted_len;
    const int64_t long_end = db->schedule == HS_SCHEDULE_INPUT ? 0 :
        std::partition_point(L.begin(), L.end(), [&](int32_t x) { return x >= long_len; }) - L.begin();
    DbView v{db->d_codes, db->d_offsets, db->d_order, db->n};
    ScanTrace tr{nullptr, nullptr};
    if (db->trace) {
        tr.start = static_cast<cudaEvent_t>(db->trace->scan_start);
        tr.stop = static_cast<cudaEvent_t>(db->trace->scan_stop);
    }
    int launches = 0;
    e = launch_prof_offsets(bl, st);
    launches++;
    if (e == cudaSuccess)
        e = launch_scan_batch(v, db->d_cumres, long_end, kp, bl, nchunk, warps, db->num_sms, d_status, st,
                              db->trace ? &tr : nullptr, &launches, db->schedule == HS_SCHEDULE_INPUT);
    if (e == cudaSuccess && nhits > 0) e = launch_topk_batch(bl, db->n, k, nhits, st, &launches);
    if (e == cudaSuccess && nhits > 0)
        e = launch_replay_batch(v, kp, bl, nhits, k, d_hits, d_ops, ops_cap, d_ops_used, d_status, st, &launches);
    if (db->trace) db->trace->launches = launches;
    return from_cuda(e);
}

int hs_search_batch(hs_db *db, int32_t nq, const uint8_t *queries, const int64_t *qoffsets, const uint64_t *seeds,
                    const hs_params *p, int32_t k, const hs_batch_tuning *tuning, void *stream, hs_hit *hits_out,
                    int32_t *n_hits_out, uint32_t *ops_out, int64_t ops_cap, int64_t *ops_used)
{
    if (!db || !p || !n_hits_out || !ops_used || nq < 0) return HS_EINVAL;
    if (nq > 0 && (!queries || !qoffsets || !seeds)) return HS_EINVAL;
    if (k < 0 || k > HS_MAX_K || ops_cap < 0) return HS_EINVAL;
    int rc = hs_params_check(p);
    if (rc != HS_OK) return rc;
    if (nq == 0) { *n_hits_out = 0; *ops_used = 0; return HS_OK; }
    if (qoffsets[0] != 0) return HS_EINVAL;
    int32_t max_qlen = 0;
    for (int32_t i = 0; i < nq; i++) {
        const int64_t ql = qoffsets[i + 1] - qoffsets[i];
        if (ql < 1) return HS_EINVAL;
        if (ql > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
        max_qlen = std::max<int32_t>(max_qlen, (int32_t)ql);
    }
    const int64_t total = qoffsets[nq];
    for (int64_t i = 0; i < total; i++)
        if (queries[i] >= kNSym) return HS_EINVAL;
    const int32_t nhits = (int32_t)std::min<int64_t>(k, db->n);
    if (nhits > 0 && !hits_out) return HS_EINVAL;

    // device/host staging: [queries | qoffsets | seeds | hits | meta | ops]
    const size_t o_q = 0, o_off = align256((size_t)total), o_seed = o_off + align256(sizeof(int64_t) * (nq + 1));
    const size_t o_hits = o_seed + align256(sizeof(uint64_t) * nq);
    const size_t o_meta = o_hits + align256(sizeof(hs_hit) * (size_t)nq * std::max(k, 1));
    const int64_t cap = hs_batch_ops_capacity(nq, total, k);
    const size_t o_ops = o_meta + 256, io_total = o_ops + align256(sizeof(uint32_t) * (size_t)std::max<int64_t>(cap, 1));
    rc = ensure_host_state(db, batch_layout(db->n, nq, total, max_qlen, k, nullptr, nullptr), io_total);
    if (rc != HS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *h = db->h_io, *d = db->d_io;
    std::memcpy(h + o_q, queries, (size_t)total);
    std::memcpy(h + o_off, qoffsets, sizeof(int64_t) * (nq + 1));
    std::memcpy(h + o_seed, seeds, sizeof(uint64_t) * nq);
    cudaError_t e = cudaMemcpyAsync(d, h, o_hits, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    rc = hs_search_batch_device(db, nq, reinterpret_cast<const uint8_t *>(d + o_q),
                                reinterpret_cast<const int64_t *>(d + o_off), reinterpret_cast<const uint64_t *>(d + o_seed),
                                total, max_qlen, p, k, tuning, stream, db->d_ws, db->ws_bytes,
                                reinterpret_cast<hs_hit *>(d + o_hits), reinterpret_cast<uint32_t *>(d + o_ops), cap,
                                reinterpret_cast<int64_t *>(d + o_meta), reinterpret_cast<int32_t *>(d + o_meta + 8));
    if (rc != HS_OK) return rc;
    // hits and status first, then only the ops actually written
    e = cudaMemcpyAsync(h + o_hits, d + o_hits, o_ops - o_hits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    int64_t used;
    int32_t status;
    std::memcpy(&used, h + o_meta, sizeof(used));
    std::memcpy(&status, h + o_meta + 8, sizeof(status));
    if (status != HS_OK) return status;
    if (nhits == 0) used = 0;
    if (used > 0) {
        e = cudaMemcpyAsync(h + o_ops, d + o_ops, sizeof(uint32_t) * (size_t)used, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (nhits > 0) std::memcpy(hits_out, h + o_hits, sizeof(hs_hit) * (size_t)nq * k);
    *n_hits_out = nhits;
    *ops_used = used;
    if (used > ops_cap) return HS_ETRUNC;
    if (used > 0) std::memcpy(ops_out, h + o_ops, sizeof(uint32_t) * (size_t)used);
    return HS_OK;
}

int hs_get_alignment(hs_db *db, const uint8_t *query, int32_t qlen, const hs_params *p, uint64_t seed,
                     int64_t db_index, void *stream, uint32_t *ops_out, int64_t cap, int32_t *score_out,
                     int64_t *ops_len_out, hs_hit *hit_out)
{
    if (!db || !query || !p || cap < 0 || (cap > 0 && !ops_out)) return HS_EINVAL;
    if (qlen < 1) return HS_EINVAL;
    if (qlen > HS_MAX_QUERY_LEN) return HS_ETOOLONG;
    db_index -= db->index_base;             // hits report global indices
    if (db_index < 0 || db_index >= db->n) return HS_EINVAL;
    for (int32_t i = 0; i < qlen; i++)
        if (query[i] >= kNSym) return HS_EINVAL;
    KParams kp;
    int rc = make_kparams(p, qlen, seed, &kp);
    if (rc != HS_OK) return rc;
    kp.s.index_base = db->index_base;
    // ops of one pair: at most 2 per step plus the tail
    const int64_t need = slot_stride_for(qlen);
    IoLayout l = io_layout(qlen, 1);
    l.total = std::max(l.total, l.ops + align256(sizeof(uint32_t) * (size_t)need));
    rc = ensure_host_state(db, workspace_bytes(db->n, qlen, 1), l.total);
    if (rc != HS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *h = db->h_io, *d = db->d_io;
    std::memcpy(h + l.q, query, (size_t)qlen);
    cudaError_t e = cudaMemcpyAsync(d + l.q, h + l.q, (size_t)qlen, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d + l.meta, 0, 16, st);
    if (e != cudaSuccess) return from_cuda(e);
    Workspace ws = carve_workspace(db->d_ws, db->n, qlen, 1);
    DbView v{db->d_codes, db->d_offsets, db->d_order, db->n};
    e = launch_replay_one(v, reinterpret_cast<const uint8_t *>(d + l.q), kp, ws, db_index,
                          reinterpret_cast<uint32_t *>(d + l.ops), need, reinterpret_cast<hs_hit *>(d + l.hits),
                          reinterpret_cast<int64_t *>(d + l.meta), reinterpret_cast<int32_t *>(d + l.meta + 8), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + l.hits, d + l.hits, l.total - l.hits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    int64_t used;
    int32_t status;
    std::memcpy(&used, h + l.meta, sizeof(used));
    std::memcpy(&status, h + l.meta + 8, sizeof(status));
    if (status != HS_OK && status != HS_ETRUNC) return status;
    hs_hit hit;
    std::memcpy(&hit, h + l.hits, sizeof(hit));
    if (score_out) *score_out = hit.score;
    if (ops_len_out) *ops_len_out = used;
    if (hit_out) *hit_out = hit;
    if (used > cap) return HS_ETRUNC;
    if (used > 0) std::memcpy(ops_out, h + l.ops, sizeof(uint32_t) * (size_t)used);
    return HS_OK;
}

}  // extern "C"
