// Host stand-in for cuda_runtime.h: lets the scan's device functions compile
// as plain C++ so CPU tests can check them.
//
// Two modes.  A thread with no warp context (lane_emu: lane-level sums and
// bounds) sees the warp-wide intrinsics as identities.  A thread that set
// emu_warp / emu_lane (pairs_emu: the whole pair loop) is one lane of a
// 32-thread warp run in lockstep: every warp intrinsic posts the lane's
// value, waits for all 32 lanes, reads what it needs and waits again, so the
// device code must call them convergently, as it must on the GPU (a lane that
// skips one leaves the others waiting, and the test times out).  A thread
// that also set emu_cta waits at __syncthreads for every thread of its CTA;
// threadIdx / blockIdx / blockDim / gridDim are per-thread variables the
// harness sets, and a kernel's __shared__ variables are function statics,
// so a harness runs one CTA at a time.
#pragma once
#define HS_HOST_EMULATION 1
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <thread>
#include <mutex>
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __align__(x) alignas(x)
#define __launch_bounds__(...)
// a kernel's shared variables: one copy, so CTAs are run one after another
#define __shared__ static
typedef int cudaError_t;
struct uint4 { unsigned x, y, z, w; };
struct alignas(8) uint2 { unsigned x, y; };
struct int2 { int x, y; };
inline int2 make_int2(int x, int y) { return int2{x, y}; }
typedef void *cudaStream_t;
typedef void *cudaEvent_t;
template <class T> inline T __ldg(const T *p) { return *p; }
inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, uint32_t sh) { return (uint32_t)((((uint64_t)hi << 32) | lo) >> (sh & 31)); }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
inline int __ffs(int x) { return __builtin_ffs(x); }
using std::min; using std::max;
// byte n of the result is byte (s >> 4n) & 7 of the 8-byte value y:x (x low)
inline uint32_t __byte_perm(uint32_t x, uint32_t y, uint32_t s) {
    uint64_t v = ((uint64_t)y << 32) | x; uint32_t r = 0;
    for (int n = 0; n < 4; n++) r |= (uint32_t)((v >> (8 * ((s >> (4 * n)) & 7))) & 0xFF) << (8 * n);
    return r;
}
// DPX maxima, as documented: the three-way unsigned maximum, and the
// maximum of two signed values with a flag telling whether the first won
// (a >= b).
inline unsigned __vimax3_u32(unsigned a, unsigned b, unsigned c) { return std::max(a, std::max(b, c)); }
inline int __vibmax_s32(int a, int b, bool *pred) { *pred = a >= b; return a >= b ? a : b; }
inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }

// ---- lockstep warp (and CTA barrier) ----------------------------------------
struct EmuBarrier {
    std::mutex mu;
    std::condition_variable cv;
    int count = 32, arrived = 0;
    uint64_t gen = 0;
    void sync() {
        std::unique_lock<std::mutex> lk(mu);
        const uint64_t g = gen;
        if (++arrived == count) {
            arrived = 0;
            gen++;
            cv.notify_all();
        } else {
            cv.wait(lk, [&] { return gen != g; });
        }
    }
};
struct EmuWarp : EmuBarrier {
    uint64_t slot[32] = {};
};
inline thread_local EmuWarp *emu_warp = nullptr;
inline thread_local int emu_lane = 0;
inline thread_local EmuBarrier *emu_cta = nullptr;     // all threads of the emulated CTA
inline void __syncthreads() { if (emu_cta) emu_cta->sync(); }
inline void __threadfence() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void __threadfence_block() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void __nanosleep(unsigned) { std::this_thread::yield(); }
// the device's global nanosecond timer
inline uint64_t emu_now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
        std::chrono::steady_clock::now().time_since_epoch()).count();
}
struct EmuDim3 { unsigned x = 0, y = 0, z = 0; };
inline thread_local EmuDim3 threadIdx, blockIdx, blockDim, gridDim;
template <class T> inline T __ldcg(const T *p) { return *p; }

template <class T> inline uint64_t emu_put(T v) { uint64_t b = 0; std::memcpy(&b, &v, sizeof(T)); return b; }
template <class T> inline T emu_get(uint64_t b) { T v; std::memcpy(&v, &b, sizeof(T)); return v; }
// every lane posts v; f reads the 32 posted words
template <class T, class F> inline auto emu_exchange(T v, F f) {
    EmuWarp &w = *emu_warp;
    w.slot[emu_lane] = emu_put(v);
    w.sync();
    auto r = f(w.slot);
    w.sync();
    return r;
}

template <class T> inline T __shfl_sync(unsigned, T v, int src) {
    if (!emu_warp) return v;
    return emu_exchange(v, [&](const uint64_t *s) { return emu_get<T>(s[src & 31]); });
}
template <class T> inline T __shfl_up_sync(unsigned, T v, unsigned d) {
    if (!emu_warp) return v;
    return emu_exchange(v, [&](const uint64_t *s) { return emu_lane >= (int)d ? emu_get<T>(s[emu_lane - d]) : v; });
}
template <class T> inline T __shfl_down_sync(unsigned, T v, unsigned d) {
    if (!emu_warp) return v;
    return emu_exchange(v, [&](const uint64_t *s) { return emu_lane + (int)d < 32 ? emu_get<T>(s[emu_lane + d]) : v; });
}
template <class T> inline T __shfl_xor_sync(unsigned, T v, int o) {
    if (!emu_warp) return v;
    return emu_exchange(v, [&](const uint64_t *s) { return emu_get<T>(s[(emu_lane ^ o) & 31]); });
}
// lanes whose value equals the calling lane's
inline unsigned __match_any_sync(unsigned, unsigned v) {
    if (!emu_warp) return 1u;
    return emu_exchange(v, [](const uint64_t *s) {
        unsigned r = 0;
        const unsigned mine = (unsigned)s[emu_lane];
        for (int i = 0; i < 32; i++) r |= ((unsigned)s[i] == mine ? 1u : 0u) << i;
        return r;
    });
}
inline unsigned __ballot_sync(unsigned, int p) {
    if (!emu_warp) return p ? 1u : 0u;
    return emu_exchange(p ? 1u : 0u, [](const uint64_t *s) {
        unsigned r = 0;
        for (int i = 0; i < 32; i++) r |= (s[i] ? 1u : 0u) << i;
        return r;
    });
}
template <class T, class Op> inline T emu_reduce(T v, Op op) {
    if (!emu_warp) return v;
    return emu_exchange(v, [&](const uint64_t *s) {
        T r = emu_get<T>(s[0]);
        for (int i = 1; i < 32; i++) r = op(r, emu_get<T>(s[i]));
        return r;
    });
}
// A reduction over the lanes named in the calling lane's mask.  Every lane
// of the warp takes part in the exchange; lanes may pass different masks
// (disjoint groups), but every lane named in a mask must have passed that
// same mask, as the hardware requires: otherwise the run aborts.
template <class T, class Op> inline T emu_reduce_masked(unsigned mask, T v, Op op) {
    static_assert(sizeof(T) == 4, "32-bit reductions");
    if (!emu_warp) return v;
    const uint64_t packed = ((uint64_t)mask << 32) | (uint64_t)(uint32_t)emu_put(v);
    return emu_exchange(packed, [&](const uint64_t *s) {
        if (!((mask >> emu_lane) & 1u)) { fprintf(stderr, "warp reduce: lane %d outside its mask\n", emu_lane); abort(); }
        T r{};
        bool first = true;
        for (int i = 0; i < 32; i++) {
            if (!((mask >> i) & 1u)) continue;
            if ((unsigned)(s[i] >> 32) != mask) { fprintf(stderr, "warp reduce: lanes of one mask disagree\n"); abort(); }
            const T x = emu_get<T>(s[i] & 0xFFFFFFFFull);
            r = first ? x : op(r, x);
            first = false;
        }
        return r;
    });
}
inline unsigned __reduce_or_sync(unsigned m, unsigned v) { return emu_reduce_masked(m, v, [](unsigned a, unsigned b) { return a | b; }); }
inline int __reduce_max_sync(unsigned m, int v) { return emu_reduce_masked(m, v, [](int a, int b) { return std::max(a, b); }); }
inline unsigned __reduce_max_sync(unsigned m, unsigned v) { return emu_reduce_masked(m, v, [](unsigned a, unsigned b) { return std::max(a, b); }); }
inline int __reduce_min_sync(unsigned m, int v) { return emu_reduce_masked(m, v, [](int a, int b) { return std::min(a, b); }); }
inline unsigned __reduce_min_sync(unsigned m, unsigned v) { return emu_reduce_masked(m, v, [](unsigned a, unsigned b) { return std::min(a, b); }); }
inline int __all_sync(unsigned, int p) { return emu_reduce(p ? 1 : 0, [](int a, int b) { return a & b; }); }
inline void __syncwarp(unsigned = 0xFFFFFFFFu) { if (emu_warp) emu_warp->sync(); }
inline unsigned atomicAdd(unsigned *p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicExch(unsigned long long *p, unsigned long long v) { return __atomic_exchange_n(p, v, __ATOMIC_SEQ_CST); }
inline int atomicCAS(int *p, int cmp, int v) {
    __atomic_compare_exchange_n(p, &cmp, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
    return cmp;
}
inline int atomicMax(int *p, int v) {
    int old = __atomic_load_n(p, __ATOMIC_SEQ_CST);
    while (old < v && !__atomic_compare_exchange_n(p, &old, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {}
    return old;
}
inline unsigned atomicMin(unsigned *p, unsigned v) {
    unsigned old = __atomic_load_n(p, __ATOMIC_SEQ_CST);
    while (old > v && !__atomic_compare_exchange_n(p, &old, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {}
    return old;
}
inline unsigned atomicMax(unsigned *p, unsigned v) {
    unsigned old = __atomic_load_n(p, __ATOMIC_SEQ_CST);
    while (old < v && !__atomic_compare_exchange_n(p, &old, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {}
    return old;
}
