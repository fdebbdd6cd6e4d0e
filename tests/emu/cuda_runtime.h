// Host stand-in for cuda_runtime.h: lets the lane-level device functions of
// the scan compile as plain C++ so a CPU test can check their sums and bounds.
// Warp-wide intrinsics are identities here; only per-lane code is exercised.
#pragma once
#include <cstdint>
#include <cstddef>
#include <algorithm>
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __align__(x) alignas(x)
typedef int cudaError_t;
struct uint4 { unsigned x, y, z, w; };
struct int2 { int x, y; };
inline int2 make_int2(int x, int y) { return int2{x, y}; }
inline void __syncthreads() {}
typedef void *cudaStream_t;
typedef void *cudaEvent_t;
template <class T> inline T __ldg(const T *p) { return *p; }
inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, uint32_t sh) { return (uint32_t)((((uint64_t)hi << 32) | lo) >> (sh & 31)); }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
using std::min; using std::max;
inline int __reduce_max_sync(unsigned, int v) { return v; }
inline int __reduce_min_sync(unsigned, int v) { return v; }
template <class T> inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
// byte n of the result is byte (s >> 4n) & 7 of the 8-byte value y:x (x low)
inline uint32_t __byte_perm(uint32_t x, uint32_t y, uint32_t s) {
    uint64_t v = ((uint64_t)y << 32) | x; uint32_t r = 0;
    for (int n = 0; n < 4; n++) r |= (uint32_t)((v >> (8 * ((s >> (4 * n)) & 7))) & 0xFF) << (8 * n);
    return r;
}
inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
