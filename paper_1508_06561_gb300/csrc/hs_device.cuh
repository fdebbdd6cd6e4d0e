// hs_device.cuh -- device building blocks of the heuristic alignment
// (Fig. 1 of Nag & Karforma, arXiv 1508.06561, in database mode, Sec. III.B.3).
//
// One warp runs one (query, target) pair.  The pair's state -- positions in
// both sequences, step, running score, the round's size factors, one cached
// random block -- is a handful of warp-uniform registers (the O(1) auxiliary
// space of Sec. III.B.4).  Inside a step the 32 lanes split the shifts of
// getBestSubsequenceAlignment: each lane owns 4 adjacent shifts packed into
// the 4 byte lanes of one 32-bit register, so one 32-bit load of the query
// profile and one integer add score 4 cells.
#pragma once
#include <climits>
#include <cstdint>

#include "hs_internal.h"

namespace hs {

// ---------------------------------------------------------------------------
// random(): Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The pair with
// database index d in round r owns 16-bit draws D_0, D_1, ...; draw i is the
// 16-bit field i%4 (most significant first) of word (i%16)/4 of the block for
// counter (d, r, i/16, 0) under key (seed, 0).  D_0 and D_1 size the round
// (lf, sf), D_(2+t) sizes step t; D / 65536 is the uniform number in [0, 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4])
{
    constexpr uint64_t kMul0 = 0xD2E7470EE14C6C93ull, kMul1 = 0xCA5A826395121157ull;
    constexpr uint64_t kWeyl0 = 0x9E3779B97F4A7C15ull, kWeyl1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; round++) {
        if (round) { k0 += kWeyl0; k1 += kWeyl1; }
        const uint64_t hi0 = __umul64hi(kMul0, c0), lo0 = kMul0 * c0;
        const uint64_t hi1 = __umul64hi(kMul1, c2), lo1 = kMul1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

struct DrawStream {
    uint64_t seed, d, r;
    int64_t blk;
    uint64_t w0, w1, w2, w3;
    __device__ __forceinline__ void init(uint64_t s, uint64_t dd, uint64_t rr)
    {
        seed = s; d = dd; r = rr; blk = -1;
    }
    __device__ __forceinline__ uint32_t get(uint64_t i)
    {
        const int64_t b = (int64_t)(i >> 4);
        if (b != blk) {
            uint64_t o[4];
            philox4x64_10(d, r, (uint64_t)b, 0, seed, 0, o);
            w0 = o[0]; w1 = o[1]; w2 = o[2]; w3 = o[3];
            blk = b;
        }
        const unsigned wi = (unsigned)(i >> 2) & 3u;
        const uint64_t w = wi == 0 ? w0 : wi == 1 ? w1 : wi == 2 ? w2 : w3;
        return (uint32_t)(w >> (48 - 16 * (unsigned)(i & 3))) & 0xFFFFu;
    }
};

// ---------------------------------------------------------------------------
// Query profile.  For role `rev` (the query is the small sequence) the
// profile holds, for every target letter a, the biased scores M[Q[.]][a] + bias
// along the reversed query; for role `fwd` (the query is the large sequence)
// along the query.  Stored column s = c + 4 (4 zero columns in front).  Word
// s of row a packs stored columns s, s+1, s+2, s+3 in its bytes 0..3, so any
// 4 consecutive columns are one aligned 32-bit load:  prof[a * R + s].
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t profile_word_value(const uint8_t *q, int qlen, bool rev,
                                                       const int8_t *m, int bias, int a, int s)
{
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int c = s + b - 4;
        uint32_t v = 0;
        if (c >= 0 && c < qlen) {
            const int qc = q[rev ? qlen - 1 - c : c];
            if (qc < kNSym) v = (uint32_t)(m[qc * kNSym + a] + bias) & 0xFFu;   // bad codes: see profile_kernel
        }
        word |= v << (8 * b);
    }
    return word;
}

// ---------------------------------------------------------------------------
// One getBestSubsequenceAlignment call in database mode (Sec. III.B.3 b):
// shifts k = 0 .. ls-ss; V(k) = sum over the ss letters of the small piece of
// M against the large piece shifted by k (the virtual score, no gaps).
//
// Work unit: a "chunk" of 4 adjacent shifts k0..k0+3 held in the 4 byte
// lanes of one register.  A chunk's cells are visited by an iteration index:
//   query large (fwd): iteration j = small letter; row = target letter
//     t[Sp+j], stored query column Lp+k0+j+4 (byte w <-> shift k0+w);
//   query small (rev): iteration p = large position relative to k0; row =
//     target letter t[Lp+k0+p], stored reversed-query column qlen+3-Sp-p;
//     byte w holds a real cell only while 0 <= p-w < ss, so iterations
//     p < 3 and p >= ss are masked (p runs over [0, ss+3)).
// Byte lanes hold biased cells (M+bias >= 0); they are widened into 32-bit
// sums every `flush` iterations, before any byte can overflow.
// ---------------------------------------------------------------------------
// Widened sums of a chunk's 4 shifts.  Acc<false>: four 32-bit sums.
// Acc<true>: two registers of two 16-bit sums each (byte w goes to half w%2
// of register w/2 by one byte permute), used when no shift's biased sum can
// reach 65536: range * (qlen + 3) <= 65535, true for BLOSUM62 at any query
// length the library accepts.
template <bool P16> struct Acc;

template <> struct Acc<false> {
    uint32_t a0, a1, a2, a3;
    __device__ __forceinline__ void zero() { a0 = a1 = a2 = a3 = 0; }
    __device__ __forceinline__ void add(uint32_t x)
    {
        a0 += x & 0xFFu;
        a1 += (x >> 8) & 0xFFu;
        a2 += (x >> 16) & 0xFFu;
        a3 += x >> 24;
    }
    __device__ __forceinline__ void xor_reduce(int o)
    {
        a0 += __shfl_xor_sync(0xFFFFFFFFu, a0, o);
        a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, o);
        a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, o);
        a3 += __shfl_xor_sync(0xFFFFFFFFu, a3, o);
    }
    __device__ __forceinline__ uint32_t get(int w) const { return w == 0 ? a0 : w == 1 ? a1 : w == 2 ? a2 : a3; }
};

template <> struct Acc<true> {
    uint32_t p01, p23;
    __device__ __forceinline__ void zero() { p01 = p23 = 0; }
    __device__ __forceinline__ void add(uint32_t x)
    {
        p01 += __byte_perm(x, 0u, 0x4140);   // bytes 0, 1 -> halves 0, 1
        p23 += __byte_perm(x, 0u, 0x4342);   // bytes 2, 3 -> halves 0, 1
    }
    __device__ __forceinline__ void xor_reduce(int o)
    {
        p01 += __shfl_xor_sync(0xFFFFFFFFu, p01, o);
        p23 += __shfl_xor_sync(0xFFFFFFFFu, p23, o);
    }
    __device__ __forceinline__ uint32_t get(int w) const
    {
        const uint32_t r = w < 2 ? p01 : p23;
        return (w & 1) ? r >> 16 : r & 0xFFFFu;
    }
};

// bytes w with w <= p and p - w < ss
__device__ __forceinline__ uint32_t edge_mask(int p, int ss)
{
    const uint32_t lo = p >= 3 ? 0xFFFFFFFFu : (0xFFFFFFFFu >> (8 * (3 - p)));
    const int h = p - ss + 1;
    const uint32_t hi = h <= 0 ? 0xFFFFFFFFu : (h >= 4 ? 0u : (0xFFFFFFFFu << (8 * h)));
    return lo & hi;
}

// Query-small iterations p in [pa, pb) of a chunk: letter tl[p], stored
// column sbase - p.  pw = prof + sbase - pa, so iteration p reads
// pw[tl[p] * R - (p - pa)].
template <bool P16>
__device__ __forceinline__ void rev_masked(const uint32_t *prof, int R, const uint8_t *tl, int sbase, int ss,
                                           int pa, int pb, int flush, Acc<P16> &A)
{
    uint32_t x = 0;
    int n = 0;
    for (int p = pa; p < pb; p++) {
        x += prof[tl[p] * R + sbase - p] & edge_mask(p, ss);
        if (++n == flush) { A.add(x); x = 0; n = 0; }
    }
    A.add(x);
}

// Sums of n iterations of a chunk: iteration j adds the profile word at
// column col0 + kDir * j in the row of letter tp[j] (kDir = -1: the query
// is small, columns of the reversed query descend; +1: the query is large).
// Four byte accumulators take a block's iterations in turn (at most flush
// each from a block of 4 * flush), eight iterations per loop trip so that a
// trip's loads issue together.
//   Rows are addressed by unsigned byte offsets from pointers bumped once
// per trip (4.3 instructions per iteration measured, against 6.6 with
// signed word indexing).
//   The scan is bound by the L1 data pipe's wavefronts (profile loads from
// shared memory plus letter loads), so the letters come as aligned 32-bit
// words -- two new words per 8 iterations -- aligned to tp by one funnel
// shift per 4 letters and split by byte permutes, instead of one byte load
// per iteration.  Words are read from tp rounded down to 4 bytes up to 11
// bytes past the last letter, inside the database's read padding.
__device__ __forceinline__ uint32_t word_at(const char *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ unsigned letter_of(uint32_t quad, int b)
{
    return __byte_perm(quad, 0u, 0x4440 + b);       // byte b of quad, zero-extended
}

template <bool P16, int kDir>
__device__ __forceinline__ void run_sums(const uint32_t *col0, int R, const uint8_t *tp, int n, int flush,
                                         Acc<P16> &A)
{
    const char *pb = reinterpret_cast<const char *>(col0);
    const unsigned R4 = 4u * (unsigned)R;
    constexpr int d = 4 * kDir;                     // bytes per iteration along the row
    const uintptr_t ta = reinterpret_cast<uintptr_t>(tp);
    const uint32_t *tw = reinterpret_cast<const uint32_t *>(ta & ~(uintptr_t)3);
    const unsigned sh = 8u * (unsigned)(ta & 3u);   // letter j sits sh bits into word pair (j/4, j/4 + 1)
    uint32_t lo = tw[0];
    for (int c = 0; c < n; c += 4 * flush) {        // blocks of 4 * flush iterations: a multiple of 4
        const int m = min(n - c, 4 * flush);
        uint32_t x = 0, y = 0, z = 0, w = 0;
        int j = 0;
        for (; j + 7 < m; j += 8) {
            const uint32_t m1 = tw[1], m2 = tw[2];
            const uint32_t q0 = __funnelshift_r(lo, m1, sh), q1 = __funnelshift_r(m1, m2, sh);
            x += word_at(pb + letter_of(q0, 0) * R4);
            y += word_at(pb + letter_of(q0, 1) * R4 + d);
            z += word_at(pb + letter_of(q0, 2) * R4 + 2 * d);
            w += word_at(pb + letter_of(q0, 3) * R4 + 3 * d);
            x += word_at(pb + letter_of(q1, 0) * R4 + 4 * d);
            y += word_at(pb + letter_of(q1, 1) * R4 + 5 * d);
            z += word_at(pb + letter_of(q1, 2) * R4 + 6 * d);
            w += word_at(pb + letter_of(q1, 3) * R4 + 7 * d);
            lo = m2;
            tw += 2;
            pb += 8 * d;
        }
        if (j + 3 < m) {
            const uint32_t m1 = tw[1];
            const uint32_t q0 = __funnelshift_r(lo, m1, sh);
            x += word_at(pb + letter_of(q0, 0) * R4);
            y += word_at(pb + letter_of(q0, 1) * R4 + d);
            z += word_at(pb + letter_of(q0, 2) * R4 + 2 * d);
            w += word_at(pb + letter_of(q0, 3) * R4 + 3 * d);
            lo = m1;
            tw += 1;
            pb += 4 * d;
            j += 4;
        }
        const int r = m - j;                        // 0 .. 3 left, only in the last block
        if (r > 0) {
            const uint32_t q0 = __funnelshift_r(lo, tw[1], sh);
            x += word_at(pb + letter_of(q0, 0) * R4);
            if (r > 1) y += word_at(pb + letter_of(q0, 1) * R4 + d);
            if (r > 2) z += word_at(pb + letter_of(q0, 2) * R4 + 2 * d);
        }
        A.add(x);
        A.add(y);
        A.add(z);
        A.add(w);
    }
}

// Unmasked query-small iterations p in [pa, pb) of a chunk: letter tl[p],
// stored column sbase - p.
template <bool P16>
__device__ __forceinline__ void rev_main(const uint32_t *prof, int R, const uint8_t *tl, int sbase, int pa,
                                         int pb, int flush, Acc<P16> &A)
{
    run_sums<P16, -1>(prof + (sbase - pa), R, tl + pa, pb - pa, flush, A);
}

// Iterations [it0, it1) of a query-small chunk, it1 - it0 >= 6 when ss >= 3.
// The segment's first 3 and last 3 iterations run with byte masks: partial
// ones where the segment holds the range's first (p < 3) or last (p >= ss)
// iterations, all-ones elsewhere -- the same instructions on every lane.
template <bool P16>
__device__ __forceinline__ void rev_segment(const uint32_t *prof, int R, const uint8_t *tl, int sbase, int ss,
                                            int it0, int it1, bool first, bool last, int flush, Acc<P16> &A)
{
    if (ss < 3) {                                   // edges overlap: mask every iteration
        rev_masked<P16>(prof, R, tl, sbase, ss, it0, it1, flush, A);
        return;
    }
    const uint32_t f0 = first ? 0x000000FFu : ~0u, f1 = first ? 0x0000FFFFu : ~0u, f2 = first ? 0x00FFFFFFu : ~0u;
    const uint32_t l0 = last ? 0xFFFFFF00u : ~0u, l1 = last ? 0xFFFF0000u : ~0u, l2 = last ? 0xFF000000u : ~0u;
    const unsigned R4 = 4u * (unsigned)R;
    const char *pf = reinterpret_cast<const char *>(prof + (sbase - it0));     // column of iteration it0
    const uint32_t a0 = word_at(pf + (unsigned)tl[it0] * R4) & f0;
    const uint32_t a1 = word_at(pf + (unsigned)tl[it0 + 1] * R4 - 4) & f1;
    const uint32_t a2 = word_at(pf + (unsigned)tl[it0 + 2] * R4 - 8) & f2;
    const int e = it1 - 3;
    const char *pl = reinterpret_cast<const char *>(prof + (sbase - e));       // column of iteration e
    const uint32_t b0 = word_at(pl + (unsigned)tl[e] * R4) & l0;
    const uint32_t b1 = word_at(pl + (unsigned)tl[e + 1] * R4 - 4) & l1;
    const uint32_t b2 = word_at(pl + (unsigned)tl[e + 2] * R4 - 8) & l2;
    if (flush >= 3) {
        A.add(a0 + a1 + a2);
        A.add(b0 + b1 + b2);
    } else {
        A.add(a0); A.add(a1); A.add(a2);
        A.add(b0); A.add(b1); A.add(b2);
    }
    if (it0 + 3 < e) rev_main<P16>(prof, R, tl, sbase, it0 + 3, e, flush, A);
}

// iterations [it0, it1) of a query-large chunk: letter ts[j], stored column
// s0 + j (no edges)
template <bool P16>
__device__ __forceinline__ void fwd_chunk(const uint32_t *prof, int R, const uint8_t *ts, int s0, int it0, int it1,
                                          int flush, Acc<P16> &A)
{
    run_sums<P16, 1>(prof + (s0 + it0), R, ts + it0, it1 - it0, flush, A);
}

__device__ __forceinline__ void lane_best1(uint32_t acc, int k, int nshift, int32_t off, int32_t &bv, int32_t &bk)
{
    const int32_t v = (int32_t)acc - off;
    bool keep;
    const int32_t m = __vibmax_s32(bv, v, &keep);      // keep: bv >= v (the earlier shift stays)
    if (k < nshift) { bk = keep ? bk : k; bv = m; }
}

// shifts ascend within a chunk, so a strict '>' keeps the lowest k
template <bool P16>
__device__ __forceinline__ void lane_best(const Acc<P16> &A, int k0, int nshift, int32_t off, int32_t &bv, int32_t &bk)
{
    lane_best1(A.get(0), k0, nshift, off, bv, bk);
    lane_best1(A.get(1), k0 + 1, nshift, off, bv, bk);
    lane_best1(A.get(2), k0 + 2, nshift, off, bv, bk);
    lane_best1(A.get(3), k0 + 3, nshift, off, bv, bk);
}

__device__ __forceinline__ void warp_argmax(int32_t bv, int32_t bk, int32_t &vmax, int32_t &kstar)
{
    vmax = __reduce_max_sync(0xFFFFFFFFu, bv);
    kstar = __reduce_min_sync(0xFFFFFFFFu, bv == vmax ? bk : INT_MAX);
}

// One step's window and its lane grid, as seen by whoever scans it.
struct __align__(16) Plan {
    const uint8_t *t;     // target letters
    int32_t Lp, Sp, ls, ss;
    int32_t qsmall;       // the query is the small sequence
    int32_t lgk, lgj;     // lane grid: 2^lgk chunks x 2^lgj segments
    int32_t pad;
};

// Lanes form a Gk x Gj grid: Gk chunks of 4 shifts side by side, each chunk's
// iterations split into Gj contiguous segments (>= 6 iterations each for
// query-small steps, whose segments carry 3 masked iterations at both ends;
// >= 4 otherwise).  Gk is the smallest power of two covering the shifts (at
// most 32, then several passes); Gj takes what the segments allow of the rest.
__device__ __forceinline__ void plan_grid(Plan &g)
{
    const int nshift = g.ls - g.ss + 1;
    const int nchunk = (nshift + 3) >> 2;
    const int lgk = nchunk >= 32 ? 5 : 32 - __clz(nchunk - 1);
    const int niter = g.qsmall ? g.ss + 3 : g.ss;
    const int minseg = g.qsmall ? 6 : 4;
    int lgj = 0;
    if (niter >= 2 * minseg) lgj = min(5 - lgk, 31 - __clz(niter / minseg));
    g.lgk = lgk;
    g.lgj = lgj;
}

// The whole warp scans one step (lane grid from plan_grid).  Byte sums of a
// chunk's segments are added across its Gj lanes by shuffles; the best
// (V, k) pair over all chunks comes from two warp reductions.
template <bool P16>
__device__ __forceinline__ void coop_scan_t(const uint32_t *prof, int R, int qlen, const Plan &g, int bias,
                                            int flush, int lane, int32_t &vmax, int32_t &kstar, int pass0 = 0,
                                            int pass_stride = 1)
{
    const int nshift = g.ls - g.ss + 1;
    const int niter = g.qsmall ? g.ss + 3 : g.ss;
    const int lgj = g.lgj;
    const int Gk = 1 << g.lgk, Gj = 1 << lgj;
    const int gk = lane >> lgj, gj = lane & (Gj - 1);
    const bool in_grid = lane < (Gk << lgj);
    const int it0 = (gj * niter) >> lgj, it1 = ((gj + 1) * niter) >> lgj;
    const int32_t off = bias * g.ss;
    const int sbase = qlen + 3 - g.Sp;
    int32_t bv = INT_MIN, bk = INT_MAX;
    for (int base = pass0 * 4 * Gk; base < nshift; base += pass_stride * 4 * Gk) {
        const int k0 = base + 4 * gk;
        const bool live = in_grid && k0 < nshift;
        Acc<P16> A;
        A.zero();
        if (live) {
            if (g.qsmall)
                rev_segment<P16>(prof, R, g.t + g.Lp + k0, sbase, g.ss, it0, it1, gj == 0, gj == Gj - 1, flush, A);
            else
                fwd_chunk<P16>(prof, R, g.t + g.Sp, g.Lp + k0 + 4, it0, it1, flush, A);
        }
        for (int o = 1; o < Gj; o <<= 1) A.xor_reduce(o);
        if (live && gj == 0) lane_best(A, k0, nshift, off, bv, bk);
    }
    warp_argmax(bv, bk, vmax, kstar);
}

__device__ __forceinline__ void coop_scan(const uint32_t *prof, int R, int qlen, const Plan &g, int bias,
                                          int flush, bool pair16, int lane, int32_t &vmax, int32_t &kstar)
{
    if (pair16) coop_scan_t<true>(prof, R, qlen, g, bias, flush, lane, vmax, kstar);
    else coop_scan_t<false>(prof, R, qlen, g, bias, flush, lane, vmax, kstar);
}

// One lane scans a whole step alone, chunk after chunk.
template <bool P16>
__device__ __forceinline__ void lane_scan_t(const uint32_t *prof, int R, int qlen, const Plan &g, int bias,
                                            int flush, int32_t &vmax, int32_t &kstar)
{
    const int nshift = g.ls - g.ss + 1;
    const int32_t off = bias * g.ss;
    int32_t bv = INT_MIN, bk = INT_MAX;
    for (int k0 = 0; k0 < nshift; k0 += 4) {
        Acc<P16> A;
        A.zero();
        if (g.qsmall) rev_segment<P16>(prof, R, g.t + g.Lp + k0, qlen + 3 - g.Sp, g.ss, 0, g.ss + 3, true, true, flush, A);
        else fwd_chunk<P16>(prof, R, g.t + g.Sp, g.Lp + k0 + 4, 0, g.ss, flush, A);
        lane_best(A, k0, nshift, off, bv, bk);
    }
    vmax = bv;
    kstar = bk;
}

__device__ __forceinline__ void lane_scan(const uint32_t *prof, int R, int qlen, const Plan &g, int bias,
                                          int flush, bool pair16, int32_t &vmax, int32_t &kstar)
{
    if (pair16) lane_scan_t<true>(prof, R, qlen, g, bias, flush, vmax, kstar);
    else lane_scan_t<false>(prof, R, qlen, g, bias, flush, vmax, kstar);
}

// One unit of the flattened scan: chunk k0..k0+3 of a step with all its
// iterations, in 16-bit pair sums.  Returns the chunk's best shift as the
// key (biased sum << 16) | (0xFFFF - k): the unsigned maximum of keys is the
// largest V with the lowest k among equals, as Fig. 1's strict '>' keeps.
// Shifts at or past nshift are left out.  Needs biased sums < 65536 (the
// 16-bit pair condition) and nshift <= 65536.  The window is given by tb
// (target letters: t + Lp when the query is small, t + Sp otherwise) and col
// (stored column base: qlen + 3 - Sp, or Lp + 4), as a flat step's
// descriptor holds them.
__device__ __forceinline__ uint32_t unit_key_at(const uint32_t *prof, int R, const uint8_t *tb, int col, int ss,
                                                bool qsmall, int k0, int nshift, int flush)
{
    Acc<true> A;
    A.zero();
    if (qsmall) rev_segment<true>(prof, R, tb + k0, col, ss, 0, ss + 3, true, true, flush, A);
    else fwd_chunk<true>(prof, R, tb, col + k0, 0, ss, flush, A);
    const uint32_t c = 0xFFFFu - (uint32_t)k0;
    const int nv = nshift - k0;                     // shifts of this chunk inside the step, >= 1
    const uint32_t y0 = __byte_perm(A.p01, c, 0x1054);   // sum of shift k0 above 0xFFFF - k0
    const uint32_t y1 = nv > 1 ? __byte_perm(A.p01, c - 1u, 0x3254) : 0u;
    const uint32_t y2 = nv > 2 ? __byte_perm(A.p23, c - 2u, 0x1054) : 0u;
    const uint32_t y3 = nv > 3 ? __byte_perm(A.p23, c - 3u, 0x3254) : 0u;
    return max(__vimax3_u32(y0, y1, y2), y3);
}

__device__ __forceinline__ uint32_t unit_key(const uint32_t *prof, int R, int qlen, const Plan &g, int k0,
                                             int nshift, int flush)
{
    return g.qsmall ? unit_key_at(prof, R, g.t + g.Lp, qlen + 3 - g.Sp, g.ss, true, k0, nshift, flush)
                    : unit_key_at(prof, R, g.t + g.Sp, g.Lp + 4, g.ss, false, k0, nshift, flush);
}

// A flat step as its units see it, 16 bytes: the target base (two words),
// stored column base | ss << 16, and (nshift - 1) | qsmall << 16.  Column
// base and ss are below 65536 because query lengths are; flat steps have
// nshift <= 65536.
__device__ __forceinline__ uint4 flat_desc(const Plan &g, int qlen)
{
    const uint8_t *tb = g.qsmall ? g.t + g.Lp : g.t + g.Sp;
    const uint32_t col = g.qsmall ? (uint32_t)(qlen + 3 - g.Sp) : (uint32_t)(g.Lp + 4);
    const uint64_t a = reinterpret_cast<uint64_t>(tb);
    uint4 d;
    d.x = (uint32_t)a;
    d.y = (uint32_t)(a >> 32);
    d.z = col | ((uint32_t)g.ss << 16);
    d.w = (uint32_t)(g.ls - g.ss) | ((uint32_t)g.qsmall << 16);
    return d;
}

__device__ __forceinline__ uint32_t desc_key(const uint32_t *prof_rev, const uint32_t *prof_fwd, int R,
                                             const uint4 &d, int k0, int flush)
{
    const uint8_t *tb = reinterpret_cast<const uint8_t *>(((uint64_t)d.y << 32) | d.x);
    const bool qsmall = (d.w >> 16) != 0;
    return unit_key_at(qsmall ? prof_rev : prof_fwd, R, tb, (int)(d.z & 0xFFFFu), (int)(d.z >> 16), qsmall, k0,
                       (int)(d.w & 0xFFFFu) + 1, flush);
}

// The bit of a pass (units base .. base + 31) where the step of one rank
// begins its units (u0), 0 if it has none or begins elsewhere.
__device__ __forceinline__ unsigned start_bit(int u0, int units, int base)
{
    const int p = u0 - base;
    return (units > 0 && p >= 0 && p < 32) ? (1u << p) : 0u;
}

// The owner (rank) of lane `lane`'s unit in a pass: the owner of the unit
// before the pass (carry; -1 before the first) plus the step beginnings at or
// below the lane (starts: the OR of the ranks' start_bit).
__device__ __forceinline__ int pass_owner(int carry, unsigned starts, int lane)
{
    return carry + __popc(starts & (0xFFFFFFFFu >> (31 - lane)));
}

// The first unit of that owner: the last beginning at or below the lane in
// this pass, else the carried owner's (carry_u0).
__device__ __forceinline__ int pass_first_unit(int carry_u0, unsigned starts, int base, int lane)
{
    const unsigned le = starts & (0xFFFFFFFFu >> (31 - lane));
    return le ? base + 31 - __clz((int)le) : carry_u0;
}

// ---------------------------------------------------------------------------
// Run-length writer for the alignment ops (lane 0 only).
// ---------------------------------------------------------------------------
struct OpWriter {
    uint32_t *out;
    int64_t cap, n, cur_len;
    uint32_t cur_op;
    __device__ __forceinline__ void init(uint32_t *o, int64_t c) { out = o; cap = c; n = 0; cur_len = 0; cur_op = 0; }
    __device__ __forceinline__ void flush()
    {
        if (cur_len > 0) {
            if (n < cap) out[n] = ((uint32_t)cur_len << 2) | cur_op;
            n++;
            cur_len = 0;
        }
    }
    __device__ __forceinline__ void push(uint32_t op, int64_t len)
    {
        if (len <= 0) return;
        if (cur_len > 0 && op == cur_op) { cur_len += len; return; }
        flush();
        cur_op = op;
        cur_len = len;
    }
};

struct Span { int32_t qb, qe, tb, te; };

// ---------------------------------------------------------------------------
// Align (Fig. 1) for one round, database mode, with the score kept
// incrementally instead of by SCORE over finished rows: every step ends in
// ss letter pairs, so its k* gap letters (in the small sequence's row) form
// one run -- periphery (PGP each) on the first step, GOP+(k*-1)GEP after --
// and the letters left when the loop ends are trailing periphery.
// Cells are counted as (ls-ss+1)*ss per step.
// ---------------------------------------------------------------------------
struct PairCtx {
    const uint32_t *prof;     // profile of this pair's role
    int S;
    const uint8_t *t;         // target letters
    int32_t tlen, qlen;
    bool qsmall;              // |T| >= |Q|: the query is the small sequence
};

template <bool EMIT>
__device__ __forceinline__ int32_t align_round(const PairCtx &c, const SParams &kp, uint64_t d, int r,
                                               int lane, int64_t &cells, OpWriter *ow, Span *span)
{
    const int32_t nl = c.qsmall ? c.tlen : c.qlen, ns = c.qsmall ? c.qlen : c.tlen;
    DrawStream ds;
    ds.init(kp.seed, d + (uint64_t)kp.index_base, (uint64_t)r);   // draws keyed by the global index
    // lf = MAX(minFactor, LFactor*random()), sf likewise (Fig. 1, Sec. III.B.1)
    uint32_t lf = (uint32_t)(((uint64_t)kp.lf_q16 * ds.get(0)) >> 16);
    uint32_t sf = (uint32_t)(((uint64_t)kp.sf_q16 * ds.get(1)) >> 16);
    lf = max(lf, kp.minf_q16);
    sf = max(sf, kp.minf_q16);
    int32_t Lp = 0, Sp = 0, score = 0;
    int64_t t = 0;
    const uint32_t gap_op = c.qsmall ? HS_OP_D : HS_OP_I;    // letters of large against gaps
    const uint32_t tail_small_op = c.qsmall ? HS_OP_I : HS_OP_D;
    while (Lp < nl && Sp < ns) {
        const int32_t Lrem = nl - Lp, Srem = ns - Sp;
        int32_t ls = (int32_t)(((uint64_t)Lrem * lf) >> 16);
        ls = max(ls, 1);
        const uint64_t u = ds.get(2 + (uint64_t)t);
        int64_t ssw = (int64_t)(((uint64_t)Srem * sf * u) >> 32);
        const int32_t ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)min(Srem, ls)));
        int32_t vmax, kstar;
        Plan g = {c.t, Lp, Sp, ls, ss, c.qsmall ? 1 : 0, 0, 0, 0};
        plan_grid(g);
        coop_scan(c.prof, c.S, c.qlen, g, kp.bias, kp.flush, kp.pair16 != 0, lane, vmax, kstar);
        cells += (int64_t)(ls - ss + 1) * ss;
        int32_t gap = 0;
        if (kstar > 0) gap = (t == 0) ? kp.pgp * kstar : kp.gop + (kstar - 1) * kp.gep;
        score += vmax - gap;
        if (EMIT && lane == 0) {
            ow->push(gap_op, kstar);
            ow->push(HS_OP_M, ss);
            const int32_t qb = c.qsmall ? Sp : Lp + kstar, tb = c.qsmall ? Lp + kstar : Sp;
            if (span->qb < 0) { span->qb = qb; span->tb = tb; }
            span->qe = qb + ss;
            span->te = tb + ss;
        }
        Lp += kstar + ss;
        Sp += ss;
        t++;
    }
    score -= kp.pgp * ((nl - Lp) + (ns - Sp));
    if (EMIT && lane == 0) {
        ow->push(gap_op, nl - Lp);
        ow->push(tail_small_op, ns - Sp);
        ow->flush();
    }
    return score;
}

// The whole CTA scans one step: warp w takes passes w, w + nw, ... of the
// lane grid, and the warps' best (V, k) pairs are reduced through shared
// memory (red: nw slots), so every thread ends with the step's argmax.
__device__ __forceinline__ void coop_scan_cta(const uint32_t *prof, int R, int qlen, const Plan &g, int bias,
                                              int flush, bool pair16, int lane, int warp, int nw, int2 *red,
                                              int32_t &vmax, int32_t &kstar)
{
    int32_t wv, wk;
    if (pair16) coop_scan_t<true>(prof, R, qlen, g, bias, flush, lane, wv, wk, warp, nw);
    else coop_scan_t<false>(prof, R, qlen, g, bias, flush, lane, wv, wk, warp, nw);
    if (lane == 0) red[warp] = make_int2(wv, wk);
    __syncthreads();
    vmax = INT_MIN;
    kstar = INT_MAX;
    for (int i = 0; i < nw; i++) {
        const int2 x = red[i];
        if (x.x > vmax || (x.x == vmax && x.y < kstar)) { vmax = x.x; kstar = x.y; }
    }
    __syncthreads();                                // red is rewritten by the next step
}

// align_round (database-search form) with every step scanned by the whole
// CTA (coop_scan_cta); all warps keep the same pair state, warp 0's lane 0
// writes the ops.  Every thread of the CTA must call it.
template <bool EMIT>
__device__ __forceinline__ int32_t align_round_cta(const PairCtx &c, const SParams &kp, uint64_t d, int r,
                                                   int lane, int warp, int nw, int2 *red, int64_t &cells,
                                                   OpWriter *ow, Span *span)
{
    const int32_t nl = c.qsmall ? c.tlen : c.qlen, ns = c.qsmall ? c.qlen : c.tlen;
    DrawStream ds;
    ds.init(kp.seed, d + (uint64_t)kp.index_base, (uint64_t)r);
    uint32_t lf = (uint32_t)(((uint64_t)kp.lf_q16 * ds.get(0)) >> 16);
    uint32_t sf = (uint32_t)(((uint64_t)kp.sf_q16 * ds.get(1)) >> 16);
    lf = max(lf, kp.minf_q16);
    sf = max(sf, kp.minf_q16);
    int32_t Lp = 0, Sp = 0, score = 0;
    int64_t t = 0;
    const bool writer = EMIT && warp == 0 && lane == 0;
    const uint32_t gap_op = c.qsmall ? HS_OP_D : HS_OP_I;
    const uint32_t tail_small_op = c.qsmall ? HS_OP_I : HS_OP_D;
    while (Lp < nl && Sp < ns) {
        const int32_t Lrem = nl - Lp, Srem = ns - Sp;
        int32_t ls = (int32_t)(((uint64_t)Lrem * lf) >> 16);
        ls = max(ls, 1);
        const uint64_t u = ds.get(2 + (uint64_t)t);
        int64_t ssw = (int64_t)(((uint64_t)Srem * sf * u) >> 32);
        const int32_t ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)min(Srem, ls)));
        int32_t vmax, kstar;
        Plan g = {c.t, Lp, Sp, ls, ss, c.qsmall ? 1 : 0, 0, 0, 0};
        plan_grid(g);
        coop_scan_cta(c.prof, c.S, c.qlen, g, kp.bias, kp.flush, kp.pair16 != 0, lane, warp, nw, red, vmax, kstar);
        cells += (int64_t)(ls - ss + 1) * ss;
        int32_t gap = 0;
        if (kstar > 0) gap = (t == 0) ? kp.pgp * kstar : kp.gop + (kstar - 1) * kp.gep;
        score += vmax - gap;
        if (writer) {
            ow->push(gap_op, kstar);
            ow->push(HS_OP_M, ss);
            const int32_t qb = c.qsmall ? Sp : Lp + kstar, tb = c.qsmall ? Lp + kstar : Sp;
            if (span->qb < 0) { span->qb = qb; span->tb = tb; }
            span->qe = qb + ss;
            span->te = tb + ss;
        }
        Lp += kstar + ss;
        Sp += ss;
        t++;
    }
    score -= kp.pgp * ((nl - Lp) + (ns - Sp));
    if (writer) {
        ow->push(gap_op, nl - Lp);
        ow->push(tail_small_op, ns - Sp);
        ow->flush();
    }
    return score;
}

// ---------------------------------------------------------------------------
// Full-slide mode (Fig. 1 as printed; readings F1-F4).  getBestSubsequence-
// Alignment slides small from overlapping large's first letter with its last
// letter to overlapping large's last letter with its first: shifts
// k = -(ss-1) .. ls-1, V(k) summed over the overlap only, lowest k on ties.
//
// The same 4-shift byte-lane chunks as the database form, from
// k0 = -(ss-1) in steps of 4; a chunk's iterations are clipped to the
// overlap and the bytes outside it are masked:
//   query small (rev): iteration p reads target letter Lp+k0+p, so the
//     window clips p to [-k0, ls-k0); byte w holds query letter Sp+p-w,
//     real while 0 <= p-w < ss (masks at p < 3 and p >= ss, as before);
//   query large (fwd): iteration j reads small letter Sp+j; byte w holds
//     query column Lp+k0+w+j, inside the window while 0 <= k0+w+j < ls
//     (masks where k0+j < 0 or k0+j+3 >= ls).
// Masked bytes add 0 and the others M + bias, so V(k) = sum - bias * (the
// overlap's length).
// ---------------------------------------------------------------------------

// bytes w with a <= w < b, of 0..3
__device__ __forceinline__ uint32_t byte_range_mask(int a, int b)
{
    const uint32_t lo = a <= 0 ? 0xFFFFFFFFu : (a >= 4 ? 0u : (0xFFFFFFFFu << (8 * a)));
    const uint32_t hi = b >= 4 ? 0xFFFFFFFFu : (b <= 0 ? 0u : (0xFFFFFFFFu >> (8 * (4 - b))));
    return lo & hi;
}

// iterations i in [i0, i1), at most 3 of them (a chunk's masked iterations
// come in runs of at most 3 at either end): row tl[i], word column
// col0 + kDir * i, bytes [a0 - kDir * i, b0 - kDir * i) kept.  Unrolled and
// predicated so that the three loads issue together.
template <bool P16, int kDir>
__device__ __forceinline__ void masked_sums(const uint32_t *prof, int R, const uint8_t *tl, int col0, int a0, int b0,
                                            int i0, int i1, int flush, Acc<P16> &A)
{
    uint32_t x = 0;
#pragma unroll
    for (int u = 0; u < 3; u++) {
        const int i = i0 + u;
        if (i < i1) {
            const uint32_t w = prof[tl[i] * R + col0 + kDir * i] & byte_range_mask(a0 - kDir * i, b0 - kDir * i);
            if (flush >= 3) x += w;             // three biased bytes fit in a byte lane
            else A.add(w);
        }
    }
    if (flush >= 3) A.add(x);
}

// Segment gj of 2^lgj (contiguous, about equal) of chunk k0's iterations.
template <bool P16>
__device__ __forceinline__ void full_chunk(const uint32_t *prof, int R, int qlen, const Plan &g, int k0, int gj,
                                           int lgj, int flush, Acc<P16> &A)
{
    const int ls = g.ls, ss = g.ss;
    int ia, ib, ca, cb;                 // iterations, and those with every byte real
    if (g.qsmall) { ia = max(0, -k0); ib = min(ss + 3, ls - k0); ca = 3; cb = ss; }
    else { ia = max(0, -k0 - 3); ib = min(ss, ls - k0); ca = -k0; cb = ls - k0 - 3; }
    const int n = ib - ia;
    const int sa = ia + ((n * gj) >> lgj), sb = ia + ((n * (gj + 1)) >> lgj);
    const int h = min(max(ca, sa), sb), e = max(min(cb, sb), h);     // [sa, h) masked, [h, e) not, [e, sb) masked
    if (g.qsmall) {
        const uint8_t *tl = g.t + g.Lp;                 // iteration p reads tl[k0 + p]
        const int sbase = qlen + 3 - g.Sp;
        masked_sums<P16, -1>(prof, R, tl + k0, sbase, 1 - ss, 1, sa, h, flush, A);
        if (e > h) run_sums<P16, -1>(prof + (sbase - h), R, tl + (k0 + h), e - h, flush, A);
        masked_sums<P16, -1>(prof, R, tl + k0, sbase, 1 - ss, 1, e, sb, flush, A);
    } else {
        const uint8_t *ts = g.t + g.Sp;
        const int s0 = g.Lp + k0 + 4;
        masked_sums<P16, 1>(prof, R, ts, s0, -k0, ls - k0, sa, h, flush, A);
        if (e > h) run_sums<P16, 1>(prof + (s0 + h), R, ts + h, e - h, flush, A);
        masked_sums<P16, 1>(prof, R, ts, s0, -k0, ls - k0, e, sb, flush, A);
    }
}

// overlap length of shift k
__device__ __forceinline__ int full_overlap(int ls, int ss, int k) { return min(ss, ls - k) - max(0, -k); }

// The whole warp scans one full-slide step: lanes form a Gk x Gj = 32 grid
// (Gk chunks side by side, each chunk's iterations split into Gj segments
// whose byte sums are added by shuffles), the shape that takes the fewest
// iteration times: passes x (iterations per segment + a pass's setup, ~8,
// and its shuffles), with segments of at least 4 iterations.
__device__ __forceinline__ int full_grid_lgk(int nchunk, int niter)
{
    int best = 5, best_cost = INT_MAX;
    for (int lk = 5; lk >= 0; lk--) {
        const int lj = 5 - lk;
        if (lj > 0 && (niter >> lj) < 4) break;       // segments only get shorter from here
        const int passes = (nchunk + (1 << lk) - 1) >> lk;
        const int cost = passes * (((niter + (1 << lj) - 1) >> lj) + 8 + 2 * lj);
        if (cost < best_cost) { best_cost = cost; best = lk; }
    }
    return best;
}

template <bool P16>
__device__ __forceinline__ void full_scan_t(const uint32_t *prof, int R, int qlen, const Plan &g, int bias, int flush,
                                            int lane, int32_t &vmax, int32_t &kstar)
{
    const int ls = g.ls, ss = g.ss;
    const int nchunk = (ls + ss - 1 + 3) >> 2;
    const int niter = g.qsmall ? ss + 3 : ss;         // the most any chunk has
    const int lgk = full_grid_lgk(nchunk, niter), lgj = 5 - lgk;
    const int Gk = 1 << lgk, Gj = 1 << lgj;
    const int gk = lane >> lgj, gj = lane & (Gj - 1);
    int32_t bv = INT_MIN, bk = INT_MAX;
    for (int c0 = 0; c0 < nchunk; c0 += Gk) {
        const int c = c0 + gk;
        const int k0 = 4 * c - (ss - 1);
        const bool live = c < nchunk;
        Acc<P16> A;
        A.zero();
        if (live) full_chunk<P16>(prof, R, qlen, g, k0, gj, lgj, flush, A);
        for (int o = 1; o < Gj; o <<= 1) A.xor_reduce(o);
        if (live && gj == 0)
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const int k = k0 + w;
                const int32_t v = (int32_t)A.get(w) - bias * full_overlap(ls, ss, k);
                if (k < ls && v > bv) { bv = v; bk = k; }      // k ascends within a lane: keeps the lowest
            }
    }
    warp_argmax(bv, bk, vmax, kstar);
}

__device__ __forceinline__ void full_scan(const uint32_t *prof, int R, int qlen, const Plan &g, int bias, int flush,
                                          bool pair16, int lane, int32_t &vmax, int32_t &kstar)
{
    if (pair16) full_scan_t<true>(prof, R, qlen, g, bias, flush, lane, vmax, kstar);
    else full_scan_t<false>(prof, R, qlen, g, bias, flush, lane, vmax, kstar);
}

// A flat full-slide step as its units see it, 16 bytes: the target base (two
// words), stored column base | ss << 16, ls | qsmall << 16.  Flat full-slide
// steps have ls + ss - 1 <= 65535, so ls, ss and k + ss - 1 fit 16 bits.
__device__ __forceinline__ uint4 full_desc(const Plan &g, int qlen)
{
    uint4 d = flat_desc(g, qlen);
    d.w = (uint32_t)g.ls | ((uint32_t)g.qsmall << 16);
    return d;
}

// The key of chunk k0 (shifts k0 .. k0 + 3 of -(ss-1) .. ls-1) of a flat
// full-slide step: the largest over its shifts k < ls of
// ((V(k) + bias * ss) << 16) | (0xFFFF - (k + ss - 1)).  V(k) + bias * ss
// lies in [0, range * ss] when the matrix has a non-negative entry (bias <=
// range), so with 16-bit pair sums it fits 16 bits; the largest key over a
// step's chunks is the best V with the lowest k (F1).
__device__ __forceinline__ uint32_t full_desc_key(const uint32_t *prof_rev, const uint32_t *prof_fwd, int R, int qlen,
                                                  const uint4 &d, int k0, int bias, int flush)
{
    Plan g;
    g.t = reinterpret_cast<const uint8_t *>(((uint64_t)d.y << 32) | d.x);
    g.qsmall = (int32_t)(d.w >> 16);
    g.ls = (int32_t)(d.w & 0xFFFFu);
    g.ss = (int32_t)(d.z >> 16);
    const int col = (int)(d.z & 0xFFFFu);
    if (g.qsmall) { g.Lp = 0; g.Sp = qlen + 3 - col; }     // tb = t + Lp, column base qlen + 3 - Sp
    else { g.Sp = 0; g.Lp = col - 4; }                      // tb = t + Sp, column base Lp + 4
    Acc<true> A;
    A.zero();
    full_chunk<true>(g.qsmall ? prof_rev : prof_fwd, R, qlen, g, k0, 0, 0, flush, A);
    uint32_t key = 0u;
#pragma unroll
    for (int w = 0; w < 4; w++) {
        const int k = k0 + w;
        const int32_t v = (int32_t)A.get(w) + bias * (g.ss - full_overlap(g.ls, g.ss, k));
        const uint32_t kw = ((uint32_t)v << 16) | (0xFFFFu - (uint32_t)(k + g.ss - 1));
        if (k < g.ls) key = max(key, kw);
    }
    return key;
}

// SCORE (reading A2) kept incrementally over the runs of a growing
// alignment, in O(1) space.  The gap runs since the last letter pair all
// share one fate: at the next letter pair they are interior (each maximal
// run of one row costs GOP+(n-1)GEP, so together runs*GOP + (gaps-runs)*GEP)
// or, if no letter pair came before them, leading periphery (PGP per gap); if
// none follows, trailing periphery (PGP per gap).  A gap run in the same row
// as the one before it extends that run.
struct RunScore {
    int32_t score, matched, last_row, runs, gaps;
    __device__ __forceinline__ void init() { score = 0; matched = 0; last_row = -1; runs = 0; gaps = 0; }
    __device__ __forceinline__ void gap(int row, int32_t n)
    {
        if (n <= 0) return;
        if (row != last_row) { runs++; last_row = row; }
        gaps += n;
    }
    __device__ __forceinline__ void match(int32_t sum, const SParams &sp)
    {
        if (!matched) score -= sp.pgp * gaps;
        else score -= runs * sp.gop + (gaps - runs) * sp.gep;
        score += sum;
        matched = 1;
        last_row = -1; runs = 0; gaps = 0;
    }
    __device__ __forceinline__ void finish(const SParams &sp)
    {
        score -= sp.pgp * gaps;
        last_row = -1; runs = 0; gaps = 0;
    }
};

template <bool EMIT>
__device__ __forceinline__ int32_t align_round_full(const PairCtx &c, const SParams &kp, uint64_t d, int r,
                                                    int lane, int64_t &cells, OpWriter *ow, Span *span)
{
    const int32_t nl = c.qsmall ? c.tlen : c.qlen, ns = c.qsmall ? c.qlen : c.tlen;
    DrawStream ds;
    ds.init(kp.seed, d + (uint64_t)kp.index_base, (uint64_t)r);
    uint32_t lf = (uint32_t)(((uint64_t)kp.lf_q16 * ds.get(0)) >> 16);
    uint32_t sf = (uint32_t)(((uint64_t)kp.sf_q16 * ds.get(1)) >> 16);
    lf = max(lf, kp.minf_q16);
    sf = max(sf, kp.minf_q16);
    int32_t Lp = 0, Sp = 0;
    int64_t t = 0;
    RunScore rs;
    rs.init();
    // ops: gaps in large's row hold small's letters, and vice versa
    const uint32_t op_gl = c.qsmall ? HS_OP_I : HS_OP_D;
    const uint32_t op_gs = c.qsmall ? HS_OP_D : HS_OP_I;
    while (Lp < nl && Sp < ns) {
        const int32_t Lrem = nl - Lp, Srem = ns - Sp;
        int32_t ls = (int32_t)(((uint64_t)Lrem * lf) >> 16);
        ls = max(ls, 1);
        const uint64_t u = ds.get(2 + (uint64_t)t);
        const int64_t ssw = (int64_t)(((uint64_t)Srem * sf * u) >> 32);
        const int32_t ss = (int32_t)max((int64_t)1, min(ssw, (int64_t)Srem));           // F2
        Plan g = {c.t, Lp, Sp, ls, ss, c.qsmall ? 1 : 0, 0, 0, 0};
        int32_t vmax, kstar;
        full_scan(c.prof, c.S, c.qlen, g, kp.bias, kp.flush, kp.pair16 != 0, lane, vmax, kstar);
        cells += (int64_t)ls * ss;           // every (window letter, piece letter) pair overlaps once
        // F3: leading overhang, overlap, trailing overhang of small
        const int32_t j0 = max(0, -kstar), j1 = min(ss, ls - kstar);
        rs.gap(0, j0);
        rs.gap(1, max(kstar, 0));
        rs.match(vmax, kp);
        rs.gap(0, ss - j1);
        if (EMIT && lane == 0) {
            ow->push(op_gl, j0);
            ow->push(op_gs, max(kstar, 0));
            ow->push(HS_OP_M, j1 - j0);
            ow->push(op_gl, ss - j1);
            const int32_t lb = Lp + kstar + j0, sb = Sp + j0;
            const int32_t qb = c.qsmall ? sb : lb, tb = c.qsmall ? lb : sb;
            if (span->qb < 0) { span->qb = qb; span->tb = tb; }
            span->qe = qb + (j1 - j0);
            span->te = tb + (j1 - j0);
        }
        Lp += kstar + j1;
        Sp += ss;
        t++;
    }
    // the end of Align (Fig. 1): large's rest against gaps in small's row, or small's rest
    rs.gap(1, nl - Lp);
    rs.gap(0, ns - Sp);
    rs.finish(kp);
    if (EMIT && lane == 0) {
        ow->push(op_gs, nl - Lp);
        ow->push(op_gl, ns - Sp);
        ow->flush();
    }
    return rs.score;
}

// AlignSequences (Fig. 1): best of `rounds` (strict '>', first best wins).
__device__ __forceinline__ int32_t align_pair(const PairCtx &c, const SParams &kp, uint64_t d, int lane,
                                              int64_t &cells, int *best_round)
{
    int32_t best = INT_MIN;
    int br = 0;
    for (int r = 0; r < kp.rounds; r++) {
        const int32_t s = kp.mode == HS_MODE_FULL ? align_round_full<false>(c, kp, d, r, lane, cells, nullptr, nullptr)
                                                  : align_round<false>(c, kp, d, r, lane, cells, nullptr, nullptr);
        if (s > best) { best = s; br = r; }
    }
    if (best_round) *best_round = br;
    return best;
}

}  // namespace hs
