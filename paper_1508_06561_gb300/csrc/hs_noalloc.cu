// hs_noalloc.cu -- a search entry point that allocates no memory.
//
// Some callers cannot allocate device memory when they search: a process
// whose memory manager reserved all device memory up front (cudaMalloc then
// fails), a latency-critical serving loop that cannot afford cudaMalloc's
// implicit device synchronisation, or a host that forbids allocation after
// start-up.  hs_search_device_noalloc serves them: its scratch lives in the
// fixed array below, part of the library's device image, so the call itself
// allocates nothing.  The caller still provides the loaded database, the
// query and every output buffer.
#include <cuda_runtime.h>

#include <mutex>

#include "hs_internal.h"

namespace {

// The scratch area.  Every GPU that loads this library holds it until the
// process exits; every call on a device shares it.
static __device__ __align__(256) unsigned char g_scratch[HS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];
void *g_scratch_ctx[kMaxDevices];       // the context the cached address belongs to

// The current context, through the driver's cuCtxGetCurrent (found once via
// the runtime, so the library links no driver library).  nullptr if unknown.
void *current_context()
{
    typedef int (*CtxGetCurrent)(void **);
    static CtxGetCurrent fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrent>(f);
    }();
    void *ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of g_scratch on the current device.  Host code only has a
// host-side stand-in for the array, so the address is looked up with
// cudaGetSymbolAddress, with the device current, once per device and
// context: a device reset (cudaDeviceReset, or the primary context torn down
// and made again) reloads the library's device image at a new address, and
// the first call after it looks the address up again.  Where the context
// cannot be read, the address is looked up on every call (the lookup
// allocates nothing).
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HS_ECUDA;
    void *ctx = current_context();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HS_ECUDA;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return HS_OK;
}

}  // namespace

extern "C" int hs_search_device_noalloc(const hs_db *db, const uint8_t *d_query, int32_t qlen,
                                        const hs_params *p, int32_t k, uint64_t seed, void *stream,
                                        hs_hit *d_hits, uint32_t *d_ops, int64_t ops_cap,
                                        int64_t *d_ops_used, int32_t *d_scores, int64_t *d_cells,
                                        int32_t *d_status)
{
    size_t need = 0;
    int rc = hs_search_workspace_size(db, qlen, k, &need);
    if (rc != HS_OK) return rc;
    if (need > (size_t)HS_NOALLOC_SCRATCH_BYTES) return HS_ETRUNC;
    void *scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != HS_OK) return rc;
    // The search clears what must start at zero (its queue counters and the
    // status word) and overwrites everything else it reads, so the previous
    // call's leftovers in the shared area do no harm.
    return hs_search_device(db, d_query, qlen, p, k, seed, stream, scratch, HS_NOALLOC_SCRATCH_BYTES, d_hits,
                            d_ops, ops_cap, d_ops_used, d_scores, d_cells, d_status);
}
